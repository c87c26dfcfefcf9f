"""GB300-native W-projection gridding and degridding (arXiv:2111.04141 hot path).

The compute path is libgw.so (CUDA kernels for sm_103a behind the C ABI in
include/gw.h); this package is its Python binding.  PyTorch is used for
device memory and streams only.
"""
from ._lib import GwError, LIB_PATH, load as load_library  # noqa: F401
from .plan import Plan, ffma_peak, launch_count  # noqa: F401
from . import hostmem  # noqa: F401

__all__ = ["Plan", "GwError", "ffma_peak", "launch_count", "load_library", "LIB_PATH"]
