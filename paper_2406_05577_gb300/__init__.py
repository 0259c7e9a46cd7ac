"""GB300-native batched, pruned plane-wave 3D FFT (sphere <-> cube).

The transform runs in libfftb.so (C ABI: include/fftb.h, CUDA kernels for
sm_103a); ``fftb`` is its ctypes binding and ``build`` compiles it in tree.
"""
from . import fftb  # noqa: F401
from .fftb import Plan, FFTBError  # noqa: F401
