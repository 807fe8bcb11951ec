"""GB300 (sm_103a) MLMC estimator of the integrated density of states of
honeycomb tight-binding sheets with random vacancies.

The compute path lives in ``libidos.so`` (CUDA kernels behind the C ABI of
``include/idos.h``); this package is a thin ctypes binding with the same
entry-point names.  Importing it loads the library and fails loudly when the
library has not been built: there is no CPU fallback.
"""
from .binding import (  # noqa: F401
    FP32_REFINE64, FP64, GRAPHENE, SMOOTH_GAUSS, SMOOTH_POLY, TMDC, IdosError, Model, Server, combine_level_stats,
    create_model, dos_from_idos, eigvalsh, fit_rates, her2k, lib_path, load_library, measure_fma_peak,
    stage1_w, status_string, tridiagonalize,
)
