"""GB300 (sm_103a) adaptive multigrid solver for the 2d Wilson-Dirac equation.

The solver (Brannick, Brower, Clark, Osborn, Rebbi, arXiv:0707.4018) runs in
hand-written CUDA kernels behind the C ABI of ``include/mg.h``; this package
holds the kernels (``csrc/``), their build (``build.py``) and a thin ctypes
binding (``binding.py``) with the same names as the C entry points.
"""
from .binding import (MG_FP16, MG_FP32, MG_FP64, CgContext, Context, half_links, half_spinor, mg_dslash_half, mg_half_convert, MGError, NullNet, autotune_report, solve_multi, load, mg_default_params, mg_dslash,  # noqa: F401
                      mg_alu_peak, mg_kernel_launches, mg_selftest_barrier, mg_smooth_fine_noalloc)
