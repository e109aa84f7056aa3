"""GB300-native HDG trace solver (Welter & Nguyen, arXiv 2512.13619).

The compute path is libhdg.so (hand-written CUDA for sm_103a behind the C ABI
of include/hdg.h).  This package holds the build script, the ctypes binding
(`_lib`, same names as the C ABI) and a thin driver that sequences the C calls
for a problem given as numpy arrays.
"""
from . import _lib  # noqa: F401
from ._lib import *  # noqa: F401,F403
