"""GB300 (sm_103a) implementation of Randomized Kaczmarz with Averaging (RKA)
and its block variant RKAB (arXiv 2401.17474) behind a C ABI
(``include/rkab.h``); this package is its thin Python binding.

The CUDA library must be built first (``build.build()``); importing the
binding's entry points raises if it is missing.  There is no CPU path.
"""
from .api import (  # noqa: F401
    Adjoint,
    AdjointConfig,
    Plan,
    RKABLstsq,
    Refiner,
    Residual,
    RkError,
    Solver,
    Spectrum,
    aligned_rows,
    alpha_star,
    launch_count,
    make_opts,
    optimal_weight,
    partial_alpha_star,
    quantize,
    rank2,
    rk_residual,
    rk_sample_indices,
    rk_setup,
    rka_solve,
    rkab_refine,
    rkab_lstsq,
    rkab_solve,
    rkab_solve_residual,
    spectrum,
    transpose,
)
