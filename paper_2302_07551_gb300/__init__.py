"""GB300-native block staircase solver for Markov-chain stationary vectors.

Python binding of libmc (include/mc.h): tensors in, device pointers out;
every step of the iteration runs in the library's CUDA kernels.  PyTorch only
provides device memory and the stream.  If libmc.so is missing this package
raises instead of falling back to anything.
"""
from ._native import McError, PLANES, load  # noqa: F401
from .chain import Chain, solve  # noqa: F401
from .server import Server  # noqa: F401
