"""GB300 (sm_103a) OEM penalized least squares for tall data.

The compute path lives in liboem.so (CUDA kernels behind the C ABI of
include/oem.h); this package is its thin Python binding. Importing it fails
if the library has not been built.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import (Context, OemError, Penalty, lib, LIB_PATH, EXPORTED, make_options,  # noqa: F401
                       oem_cv, oem_fit, oem_fit_path, oem_fold_grams, oem_gram, oem_spectral_d)
