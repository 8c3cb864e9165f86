"""GB300 (sm_103a) hot path of the TACAW method (arXiv 2401.15599).

The computation lives in libtacaw.so (C-ABI in include/tacaw.h); ``api``
wraps it for PyTorch tensors.  Importing this package loads nothing; the
library is loaded (and must exist) on the first call.
"""

__all__ = ["api", "build"]
