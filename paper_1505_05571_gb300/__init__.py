"""Exact FP64 summation on GB300 (small and large superaccumulators, Neal 2015).

The compute path is the CUDA library ``libxsum.so`` (C ABI in include/xsum.h);
``xsum`` is its ctypes binding and ``build`` compiles it in-tree for sm_103a.
"""

from . import xsum  # noqa: F401
from .xsum import *  # noqa: F401,F403
