"""GB300 (sm_103a) library for the second-kind integral equations of the 2D
elastance and mobility problems (Rachh & Greengard, arXiv:1507.05925).

The compute path is the CUDA library libbie2d (C ABI in include/bie2d.h);
``bie`` is its thin ctypes binding, ``build`` compiles it in-tree.
"""
from .bie import (  # noqa: F401
    ERR_CUDA, ERR_INVALID, ERR_NOMEM, ERR_OUTSIDE, FP64, LAPLACE, MIXED, MIXED_FF, OK, STOKES,
    WARN_NONNEUTRAL, WARN_NOT_CONVERGED, Context, apply_operator, elastance_solve, elastance_solve_batch,
    make_opts, mobility_solve, mobility_solve_batch, tune, tune_clear,
)
