"""GB300-native Stochastic Bundle Adjustment: the LM iteration hot path as a C-ABI CUDA library.

`stba` is the ctypes binding of libstba.so (see include/stba.h for the contract)."""
from . import stba  # noqa: F401
from .stba import Context, StbaError  # noqa: F401
