"""GB300-native velocity-gauge RT-TDDFT step in an auxiliary subspace.

The compute path is the CUDA library librttddft.so (C ABI in
include/rttddft.h); `rttddft` binds it with ctypes.  There is no CPU
fallback: calls fail if the library is not built or no GPU is present.
"""
from .build import LIB_PATH, build
from . import rttddft
from .rttddft import Context, RttddftError, load_library

__all__ = ["LIB_PATH", "build", "rttddft", "Context", "RttddftError", "load_library"]
