"""GB300-native (sm_103a) unfitted boundary algebraic equation solver with
lattice Green's functions (Xia, arXiv 2502.05507).

The computation lives in libbae.so (CUDA, C ABI in include/bae.h); this
package holds its sources (csrc/), the build script and a ctypes binding.
"""
from .bae import (BAEError, Context, GeometryError, NotConverged, Problem, lib, FP32, FP64, MIXED, DF64,  # noqa: F401
                  LAYER_DOUBLE, LAYER_SINGLE, EXPORTED, Server, launch_count, profile_start, profile_stop,
                  set_conv_schedule)
