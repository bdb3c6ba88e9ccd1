"""GB300 (sm_103a) hierarchical Hough transform for straight lines.

The package holds the CUDA library (csrc/, built into _build/libhht.so by
build.py) and its thin Python binding (hht.py).  See include/hht.h for the
C ABI.
"""
from . import hht  # noqa: F401
from .hht import Context, Result, HhtError, detect, load, version  # noqa: F401
