"""GB300-native energy-aware auto-tuning of an FP32 2-D convolution.

The compute path is ``libconvtune.so`` (hand-written CUDA for sm_103a plus a
C++ runtime behind the C-ABI in ``include/convtune.h``); ``api`` is a thin
ctypes binding to it.  Importing this package loads nothing; the library is
loaded on first use and its absence is an error, never a fallback.
"""
__all__ = ["api", "synth"]
