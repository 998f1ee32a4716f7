"""GB300-native velocity-gauge RT-TDDFT step in an auxiliary subspace.

The compute path is the CUDA library librttddft.so (C ABI in
include/rttddft.h); `rttddft` binds it with ctypes.  There is no CPU
fallback: calls fail if the library is not built or no GPU is present.
"""
from .build import LIB_PATH, build
from . import rttddft
from .rttddft import Context, RttddftError, load_library


def dipole_increment(a_samples, context, ckpt_every=50):
    """dmu(t0 + n dt) - dmu(t0) of `context`'s run over the pulse samples, differentiable
    with respect to the samples (torch.autograd; see `autograd.DipoleIncrement`)."""
    from .autograd import DipoleIncrement
    return DipoleIncrement.apply(a_samples, context, ckpt_every)


__all__ = ["LIB_PATH", "build", "rttddft", "Context", "RttddftError", "load_library", "dipole_increment"]
