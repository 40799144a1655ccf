"""GB300-native spin-1 Bogoliubov-de Gennes excitation solver (Fourier spectral
method of arXiv 2506.08308): a CUDA library with a C ABI (include/bdg.h) and
this thin Python binding."""
from .bdg import (C64, C128, FG, FP64, MIXED, UV, BdgError, Plan, ground_state, load,  # noqa: F401
                  make_params, params_from)
