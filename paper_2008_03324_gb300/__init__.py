"""GB300-native Fisher Information Field (arXiv 2008.03324): field build and pose query.

The compute path is the in-tree CUDA library ``libfif.so`` (hand-written kernels for
sm_103a behind a C ABI, declared in ``include/fif.h``).  :mod:`.fif` is a thin ctypes
binding with the same names; it raises if the library is missing -- there is no CPU
fallback.  :mod:`.synth` draws the seeded synthetic inputs.
"""
__all__ = ["synth"]
