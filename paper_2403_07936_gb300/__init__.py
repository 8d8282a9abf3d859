"""GB300-native periodic multigrid V-cycle with cubic and super-resolution
prolongation (arXiv 2403.07936), behind the C ABI of include/mg.h.

The compute path is libmg.so (hand-written CUDA for sm_103a); this package is
its build script and a thin ctypes binding.
"""
from . import mg  # noqa: F401
from .mg import Context, MGError, load, solve_batched  # noqa: F401
