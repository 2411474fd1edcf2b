"""GB300 (sm_103a) implementation of the VaFR ray-casting hot path.

The computation lives in libvafr.so (CUDA kernels behind the C ABI declared in
include/vafr.h); ``vafr`` is its ctypes binding and ``serve`` the
continuous-batching request loop built on it.  PyTorch is used only for device
memory and streams.
"""

from . import vafr  # noqa: F401
from .vafr import VafrError  # noqa: F401

__all__ = ["vafr", "VafrError"]
