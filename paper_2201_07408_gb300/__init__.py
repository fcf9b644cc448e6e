"""GB300 (sm_103a) CUDA library for CT reconstruction with an unmatched
projector/back-projector pair by BA-GMRES / AB-GMRES (arXiv 2201.07408).

The compute path is libct.so (C-ABI, include/ct.h); ``ct`` is its ctypes
binding and ``autograd`` wraps it in torch.autograd Functions.
"""
from . import ct  # noqa: F401
from .ct import Geometry, CTError  # noqa: F401

__all__ = ["ct", "Geometry", "CTError"]
