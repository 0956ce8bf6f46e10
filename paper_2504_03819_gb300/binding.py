"""Thin ctypes binding of the C ABI in include/lbm.h.

Argument marshalling only: every step of the model runs in the CUDA kernels of
liblbm.so.  PyTorch provides device memory and the CUDA stream.  There is no
CPU fallback: if the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_STATE, LBM_ERR_NONFINITE, LBM_ERR_DOMAIN, LBM_ERR_SIZE = \
    0, -1, -2, -3, -4, -5, -6
LBM_ERR_TIMEOUT = -7
LBM_F32, LBM_F16 = 0, 1
SHIFT_CONST, SHIFT_REST = 0, 1
WET_NEUTRAL, WET_PHI, WET_DELTA = 0, 1, 2
OBJ_ENERGY, OBJ_CENTROID_X, OBJ_CONTACT_RADIUS = 0, 1, 2
NGRAD = 13   # [kappa, omega_0 .. omega_10, wetting_value]
ERROR_NAMES = {LBM_ERR_ARG: "LBM_ERR_ARG", LBM_ERR_CUDA: "LBM_ERR_CUDA", LBM_ERR_STATE: "LBM_ERR_STATE",
               LBM_ERR_NONFINITE: "LBM_ERR_NONFINITE", LBM_ERR_DOMAIN: "LBM_ERR_DOMAIN",
               LBM_ERR_SIZE: "LBM_ERR_SIZE", LBM_ERR_TIMEOUT: "LBM_ERR_TIMEOUT"}

# Every symbol include/lbm.h declares, with (restype, argtypes).
SIGNATURES = {
    "lbm_workspace_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int]),
    "lbm_init_domain": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_size_t, C.c_void_p]),
    "lbm_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_wall_velocity": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_sync_status": (C.c_int, [C.c_void_p]),
    "lbm_inject_wait_timeout": (C.c_int, [C.c_void_p]),
    "lbm_set_fused_moments": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_stored_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_status_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_state_bytes": (C.c_size_t, [C.c_void_p]),
    "lbm_get_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_raw_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_get_populations": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_set_populations": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lbm_objective": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_adjoint_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_adjoint_pool_bytes": (C.c_size_t, [C.c_void_p]),
    "lbm_adjoint_segment": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "lbm_adjoint_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_destroy": (None, [C.c_void_p]),
    "lbm_launch_count": (C.c_longlong, [C.c_void_p]),
    "lbm_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "lbm_kernel_name": (C.c_char_p, [C.c_int]),
    "lbm_step_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                   C.c_void_p]),
    "lbm_maxwell": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                              C.POINTER(C.c_double)]),
}


class LbmParams(C.Structure):
    """Mirror of lbm_params (include/lbm.h)."""
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("T", C.c_double),
                ("kappa", C.c_double), ("omega", C.c_double * 11), ("nu", C.c_double),
                ("q4_correction", C.c_int), ("wetting_mode", C.c_int), ("wetting_value", C.c_double),
                ("rho_l", C.c_double), ("rho_v", C.c_double), ("rho_shift", C.c_double),
                ("shift_mode", C.c_int), ("check_interval", C.c_int)]


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load() -> C.CDLL:
    """Load liblbm.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def maxwell(a: float, b: float, R: float, T: float) -> tuple[float, float]:
    """Coexistence densities (rho_l, rho_v) from the library's host helper."""
    rl, rv = C.c_double(), C.c_double()
    rc = load().lbm_maxwell(a, b, R, T, C.byref(rl), C.byref(rv))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_maxwell: T must be below T_c and a, b, R > 0")
    return rl.value, rv.value


@dataclass
class Params:
    """Model parameters (field meanings as in lbm_params)."""
    a: float
    b: float
    R: float
    T: float
    kappa: float
    omega: list = field(default_factory=lambda: [1.0] * 11)
    nu: float = 0.0
    q4_correction: int = 1
    wetting_mode: int = WET_NEUTRAL
    wetting_value: float = 1.0
    rho_l: float = 0.0
    rho_v: float = 0.0
    rho_shift: float = 0.0
    shift_mode: int = SHIFT_REST
    check_interval: int = 0

    @staticmethod
    def vdw(a: float, b: float, R: float, t_over_tc: float, kappa: float, **kw) -> "Params":
        """Parameters at T = t_over_tc * T_c with T_c = 8a/(27Rb) (Eq. 30);
        rho_l, rho_v from the Maxwell construction unless given."""
        T = t_over_tc * 8.0 * a / (27.0 * R * b)
        if "rho_l" not in kw or "rho_v" not in kw:
            kw["rho_l"], kw["rho_v"] = maxwell(a, b, R, T)
        return Params(a=a, b=b, R=R, T=T, kappa=kappa, **kw)

    def to_c(self, storage: int = LBM_F32) -> LbmParams:
        p = LbmParams()
        p.shift_mode = int(self.shift_mode)
        for name in ("a", "b", "R", "T", "kappa", "nu", "wetting_value", "rho_l", "rho_v", "rho_shift"):
            setattr(p, name, float(getattr(self, name)))
        for i in range(11):
            p.omega[i] = float(self.omega[i])
        p.q4_correction = int(self.q4_correction)
        p.wetting_mode = int(self.wetting_mode)
        p.check_interval = int(self.check_interval)
        return p


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


NOALLOC_MAX_NODES = 32768


def step_noalloc(f_in, f_out, solid_mask, params: Params, stream=None) -> int:
    """One step through lbm_step_noalloc, for callers that cannot allocate
    device memory (the library keeps the scratch in a static device array).
    f_in, f_out: CUDA float32 tensors (27, nz, ny, nx); solid_mask: CUDA uint8
    (nz, ny, nx) or None.  Returns the LBM_* status code."""
    import torch
    for name, t in (("f_in", f_in), ("f_out", f_out), ("solid_mask", solid_mask)):
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor (no copy is made)")
    if f_in.dtype != torch.float32 or f_out.dtype != torch.float32 or f_in.shape != f_out.shape:
        raise ValueError("f_in and f_out must be float32 tensors of the same shape (27, nz, ny, nx)")
    _, nz, ny, nx = f_in.shape
    pc = params.to_c()
    s = stream if stream is not None else torch.cuda.current_stream(f_in.device)
    return load().lbm_step_noalloc(_ptr(f_in), _ptr(f_out), _ptr(solid_mask), nx, ny, nz, C.byref(pc),
                                   C.c_void_p(s.cuda_stream))


class Domain:
    """One simulation domain on one GPU: the C-ABI context plus the torch
    tensors (workspace, solid mask) whose memory it views.

    Field tensors are laid out (nz, ny, nx); vector fields (3, nz, ny, nx);
    populations (27, nz, ny, nx) with q = (cx+1) + 3(cy+1) + 9(cz+1).
    """

    def __init__(self, nx: int, ny: int, nz: int, storage: str = "f32", solid_mask=None,
                 device: str = "cuda", stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the library has no CPU path")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.storage = {"f32": LBM_F32, "f16": LBM_F16}[storage]
        self.pop_dtype = torch.float32 if self.storage == LBM_F32 else torch.float16
        self.device = torch.device(device)
        nbytes = self.lib.lbm_workspace_bytes(nx, ny, nz, self.storage)
        if nbytes == 0:
            raise LbmError(LBM_ERR_SIZE, "invalid domain size")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.mask = None
        if solid_mask is not None:
            self.mask = torch.as_tensor(solid_mask).to(device=self.device, dtype=torch.uint8).contiguous()
            assert self.mask.numel() == self.N
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = C.c_void_p()
        rc = self.lib.lbm_init_domain(C.byref(ctx), nx, ny, nz, self.storage, _ptr(self.mask),
                                      _ptr(self.workspace), nbytes, C.c_void_p(self.stream.cuda_stream))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_init_domain failed")
        self.ctx = ctx

    # -- helpers -------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != LBM_OK:
            raise LbmError(rc, f"{what}: {self.lib.lbm_last_error(self.ctx).decode()}")

    def _dev(self, x, shape, dtype=None):
        t = self.torch
        dtype = dtype or t.float32
        x = t.as_tensor(x)
        x = x.to(device=self.device, dtype=dtype).contiguous()
        assert tuple(x.shape) == tuple(shape), (x.shape, shape)
        return x

    # -- API -------------------------------------------------------------------
    def set_params(self, p: Params):
        self._params_c = p.to_c(self.storage)
        self.params = p
        self._check(self.lib.lbm_set_params(self.ctx, C.byref(self._params_c)), "lbm_set_params")

    def set_wall_velocity(self, wall_u=None):
        """Velocities of the solid nodes, shape (3, nz, ny, nx) (values on
        fluid nodes unused), or None for walls at rest.  The device copy is
        kept alive by the domain."""
        if wall_u is None:
            self._wall_u = None
            ptr = None
        else:
            self._wall_u = self._dev(wall_u, (3, self.nz, self.ny, self.nx))
            ptr = _ptr(self._wall_u)
        self._check(self.lib.lbm_set_wall_velocity(self.ctx, ptr), "lbm_set_wall_velocity")

    def set_state(self, rho0, u0=None):
        shp = (self.nz, self.ny, self.nx)
        r = self._dev(rho0, shp)
        u = None if u0 is None else self._dev(u0, (3,) + shp)
        self._check(self.lib.lbm_set_state(self.ctx, _ptr(r), _ptr(u)), "lbm_set_state")
        self.stream.synchronize()

    def step(self, n: int = 1):
        self._check(self.lib.lbm_step(self.ctx, int(n)), "lbm_step")

    def sync_status(self) -> int:
        return self.lib.lbm_sync_status(self.ctx)

    def fuse_moments(self, on: bool = True):
        """Opt-in step variant: the fused kernel also forms the next state's
        moments (lbm_set_fused_moments)."""
        self._check(self.lib.lbm_set_fused_moments(self.ctx, 1 if on else 0), "lbm_set_fused_moments")

    def stored_moments(self) -> dict:
        """The moments the next step starts from, as stored (rho, j, mu0 - mu_ref;
        lbm_stored_moments)."""
        t = self.torch
        rho = t.empty((self.nz, self.ny, self.nx), dtype=t.float32, device=self.device)
        j = t.empty((3, self.nz, self.ny, self.nx), dtype=t.float32, device=self.device)
        mu0 = t.empty_like(rho)
        self._check(self.lib.lbm_stored_moments(self.ctx, _ptr(rho), _ptr(j), _ptr(mu0)), "lbm_stored_moments")
        return {"rho": rho, "j": j, "mu0": mu0}

    def inject_wait_timeout(self):
        """Failure-path test hook: the next step's fused kernel lets one
        bounded wait run out (lbm_inject_wait_timeout)."""
        self._check(self.lib.lbm_inject_wait_timeout(self.ctx), "lbm_inject_wait_timeout")

    def status_async(self, out):
        """Enqueue a copy of the status word into `out` (a pinned int32 CPU
        tensor with at least one element) and return at once; once the stream
        has reached it, out[0] != 0 means a flag is set (sync_status gives the
        code)."""
        t = self.torch
        if out.device.type != "cpu" or out.dtype != t.int32 or out.numel() < 1:
            raise ValueError("status_async needs an int32 CPU tensor")
        self._check(self.lib.lbm_status_async(self.ctx, C.c_void_p(out.data_ptr())), "lbm_status_async")

    def moments(self) -> dict:
        t = self.torch
        shp = (self.nz, self.ny, self.nx)
        rho = t.empty(shp, dtype=t.float32, device=self.device)
        mu = t.empty(shp, dtype=t.float32, device=self.device)
        u = t.empty((3,) + shp, dtype=t.float32, device=self.device)
        me = t.empty(2, dtype=t.float64, device=self.device)
        self._check(self.lib.lbm_moments(self.ctx, _ptr(rho), _ptr(u), _ptr(mu), _ptr(me)), "lbm_moments")
        self.stream.synchronize()
        return dict(rho=rho, u=u, mu=mu, mass=float(me[0]), energy=float(me[1]))

    def state_bytes(self) -> int:
        return int(self.lib.lbm_state_bytes(self.ctx))

    def get_state(self, out=None, sync: bool = True):
        """Raw state as a flat uint8 device tensor (lbm_state_bytes bytes)."""
        t = self.torch
        if out is None:
            out = t.empty(self.state_bytes(), dtype=t.uint8, device=self.device)
        self._check(self.lib.lbm_get_state(self.ctx, _ptr(out)), "lbm_get_state")
        if sync:
            self.stream.synchronize()
        return out

    def set_raw_state(self, raw, sync: bool = True):
        raw = raw.to(device=self.device, dtype=self.torch.uint8).contiguous()
        assert raw.numel() == self.state_bytes()
        self._check(self.lib.lbm_set_raw_state(self.ctx, _ptr(raw)), "lbm_set_raw_state")
        if sync:
            self.stream.synchronize()

    def get_populations(self):
        t = self.torch
        out = t.empty((27, self.nz, self.ny, self.nx), dtype=t.float32, device=self.device)
        self._check(self.lib.lbm_get_populations(self.ctx, _ptr(out)), "lbm_get_populations")
        self.stream.synchronize()
        return out

    def set_populations(self, f):
        f = self._dev(f, (27, self.nz, self.ny, self.nx))
        self._check(self.lib.lbm_set_populations(self.ctx, _ptr(f)), "lbm_set_populations")
        self.stream.synchronize()

    # -- discrete adjoint -------------------------------------------------------
    def objective(self, kind: int, wall_z: int = 0, grad=None):
        """(J, dJ/df) of the current state; J is a CUDA float64 tensor (2,).
        The objective's direct parameter dependence is added to grad if given."""
        t = self.torch
        J = t.zeros(2, dtype=t.float64, device=self.device)
        lam = t.empty((27, self.nz, self.ny, self.nx), dtype=t.float32, device=self.device)
        self._check(self.lib.lbm_objective(self.ctx, int(kind), int(wall_z), _ptr(J), _ptr(lam), _ptr(grad)),
                    "lbm_objective")
        return J, lam

    def adjoint_step(self, state_t, lam_next, grad, lam_out=None):
        """dJ/df(t) from dJ/df(t+1) at the raw state of time t; adds the
        parameter gradients to grad (CUDA float64, NGRAD)."""
        t = self.torch
        lam_next = self._dev(lam_next, (27, self.nz, self.ny, self.nx))
        out = lam_out if lam_out is not None else t.empty_like(lam_next)
        raw = state_t.to(device=self.device, dtype=t.uint8).contiguous()
        assert raw.numel() == self.state_bytes() and grad.dtype == t.float64 and grad.numel() == NGRAD
        self._check(self.lib.lbm_adjoint_step(self.ctx, _ptr(raw), _ptr(lam_next), _ptr(out), _ptr(grad)),
                    "lbm_adjoint_step")
        return out

    def adjoint_pool_bytes(self) -> int:
        """Bytes per step of the adjoint_segment pool (raw state + captured fields)."""
        return int(self.lib.lbm_adjoint_pool_bytes(self.ctx))

    def adjoint_segment(self, ckpt, n: int, pool, lam, lam_tmp, grad):
        """In place: lam = dJ/df(t0+n) -> dJ/df(t0) over the n steps after the
        raw checkpoint ckpt; pool holds >= n * adjoint_pool_bytes() bytes
        (uint8, CUDA)."""
        assert pool.numel() >= n * self.adjoint_pool_bytes() and grad.numel() == NGRAD
        self._check(self.lib.lbm_adjoint_segment(self.ctx, _ptr(ckpt), int(n), _ptr(pool), _ptr(lam),
                                                 _ptr(lam_tmp), _ptr(grad)), "lbm_adjoint_segment")
        return lam

    def adjoint_init(self, rho0, u0, lam0, grad):
        """dJ/drho0 from dJ/df(0); adds the initialisation's parameter
        gradients to grad.  Leaves the initial state of rho0, u0 current."""
        t = self.torch
        shp = (self.nz, self.ny, self.nx)
        r = self._dev(rho0, shp)
        u = None if u0 is None else self._dev(u0, (3,) + shp)
        lam0 = self._dev(lam0, (27,) + shp)
        g = t.empty(shp, dtype=t.float32, device=self.device)
        self._check(self.lib.lbm_adjoint_init(self.ctx, _ptr(r), _ptr(u), _ptr(lam0), _ptr(grad), _ptr(g)),
                    "lbm_adjoint_init")
        return g

    def launch_count(self) -> int:
        return int(self.lib.lbm_launch_count(self.ctx))

    def profile(self, on: bool):
        self._check(self.lib.lbm_profile_enable(self.ctx, 1 if on else 0), "lbm_profile_enable")

    def profile_read(self) -> dict:
        out = {}
        i = 0
        while True:
            name = self.lib.lbm_kernel_name(i)
            if name is None:
                break
            ms, n = C.c_double(), C.c_longlong()
            self._check(self.lib.lbm_profile_read(self.ctx, i, C.byref(ms), C.byref(n)), "lbm_profile_read")
            out[name.decode()] = (ms.value, n.value)
            i += 1
        return out

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
