"""GB300-native revectorization-based shadow mapping (RBSM) visibility.

The compute lives in librbsm.so (hand-written sm_103a CUDA behind the C ABI
of include/rbsm.h).  This package holds that library's sources and build
step (``build``), its ctypes description (``_native``) and a thin torch
binding with the ABI's names (``api``).
"""
from . import _native  # noqa: F401  (no library load at import time)

__all__ = ["api", "build", "_native"]
