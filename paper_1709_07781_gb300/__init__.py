"""Order-preserving stream compaction as composed kernel actors on GB300.

The library is libka.so (CUDA kernels for sm_103a plus the actor runtime, C
ABI in include/ka.h); this package is its ctypes binding (`_lib`, same names
as the C entry points) and its build script (`build`).
"""
from . import _lib  # noqa: F401  (raises ImportError when libka.so is not built)
from ._lib import *  # noqa: F401,F403
