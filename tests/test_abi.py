"""The C-ABI library loads and exports every symbol include/lbm.h declares;
host-only entry points validate their arguments (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

import __graft_entry__
from oracle import thermo as T
from paper_2504_03819_gb300 import binding as Bd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return Bd.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(Bd.SIGNATURES), set(names) ^ set(Bd.SIGNATURES)


def test_params_struct_layout_matches_header():
    # 5 doubles, 11 doubles, nu, 2 ints, 3 doubles, rho_shift, 2 ints
    assert C.sizeof(Bd.LbmParams) == 8 * 5 + 8 * 11 + 8 + 4 + 4 + 8 * 3 + 8 + 4 + 4


def test_workspace_bytes_and_argument_checks(lib):
    n = lib.lbm_workspace_bytes(16, 8, 4, Bd.LBM_F32)
    N = 16 * 8 * 4
    assert n >= 2 * 27 * N * 4 + 17 * N * 4 and n % 256 == 0
    assert lib.lbm_workspace_bytes(16, 8, 4, Bd.LBM_F16) < n
    assert lib.lbm_workspace_bytes(0, 8, 4, Bd.LBM_F32) == 0
    assert lib.lbm_workspace_bytes(4, 4, 4, 7) == 0
    assert lib.lbm_workspace_bytes(2048, 2048, 1024, Bd.LBM_F32) == 0  # N >= 2^31
    ctx = C.c_void_p()
    assert lib.lbm_init_domain(C.byref(ctx), 0, 4, 4, 0, None, None, 0, None) == Bd.LBM_ERR_ARG
    assert lib.lbm_init_domain(C.byref(ctx), 4, 4, 4, 0, None, None, 0, None) == Bd.LBM_ERR_ARG
    assert lib.lbm_init_domain(C.byref(ctx), 4, 4, 4, 0, None, C.c_void_p(256), 16, None) == Bd.LBM_ERR_SIZE
    assert lib.lbm_init_domain(None, 4, 4, 4, 0, None, None, 0, None) == Bd.LBM_ERR_ARG
    assert lib.lbm_step(None, 1) == Bd.LBM_ERR_ARG
    assert lib.lbm_set_params(None, None) == Bd.LBM_ERR_ARG
    assert lib.lbm_last_error(None) == b"null context"
    assert lib.lbm_kernel_name(0) is not None and lib.lbm_kernel_name(999) is None


@pytest.mark.parametrize("a,t", [(9 / 392, 0.7), (9 / 49, 0.85), (9 / 49, 0.6), (9 / 392, 0.95)])
def test_library_maxwell_matches_oracle(lib, a, t):
    eos = T.at_reduced_temperature(a, 2 / 21, 1.0, t)
    rl, rv = Bd.maxwell(a, 2 / 21, 1.0, eos.T)
    ol, ov = T.maxwell(eos)
    assert rl == pytest.approx(ol, rel=1e-12) and rv == pytest.approx(ov, rel=1e-10)


def test_library_maxwell_rejects_supercritical(lib):
    with pytest.raises(Bd.LbmError):
        Bd.maxwell(9 / 49, 2 / 21, 1.0, 1.01 * 8 * (9 / 49) / (27 * 2 / 21))
