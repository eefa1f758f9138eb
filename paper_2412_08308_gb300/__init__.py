"""GB300-native score-only Smith-Waterman/Gotoh protein database search.

The computation lives in the CUDA library ``libswgb.so`` behind the C-ABI of
``include/swgb.h``; this package is the thin Python side: ``_native`` (ctypes,
same names as the C entry points) and ``api`` (numpy / torch marshalling).
PyTorch is used only for device memory and streams.
"""

from . import api  # noqa: F401
from .build import build  # noqa: F401

__all__ = ["build", "api"]
