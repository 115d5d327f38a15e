"""FP64 CPU oracle for the fully discrete third-order Active Flux method
(arXiv 2508.06273) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never does, and the
oracle imports nothing from the library.
"""
from .afo import (  # noqa: F401
    Oracle,
    build,
    correction_T,
    eg_field,
    set_quadrature,
    VTX,
    XE,
    YE,
    BC_PERIODIC,
    BC_TRANSMISSIVE,
    BC_REFLECTING,
    BC_INFLOW,
    OPT_LIN_MODE,
    OPT_TSW,
    OPT_LIMITER,
    OPT_CORRECTION,
    OPT_FORCE_LO,
    OPT_THREADS,
    OPT_FLUX_LIMITER,
    OPT_SHOCK_BLEND,
    OPT_NODE_BOUNDS,
    OPT_UBAR,
    ST_FLUX_LIMITED,
    ST_CFL,
    ST_AVG_NONPOS,
    ST_NONFINITE,
    ST_KEPT,
)
