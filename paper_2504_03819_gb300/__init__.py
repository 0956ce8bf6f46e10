"""GB300-native free-energy D3Q27 lattice Boltzmann hot path (arXiv 2504.03819).

The compute path is liblbm.so (hand-written CUDA for sm_103a behind the C ABI of
include/lbm.h); ``binding`` is its thin ctypes wrapper and ``inputs`` builds the
seeded synthetic initial conditions.  Importing the package does not load the
library; ``binding.load()`` (or creating a ``Domain``) does, and raises if it
is not built.
"""
from .binding import Domain, LbmError, Params, load, maxwell  # noqa: F401
