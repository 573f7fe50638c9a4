"""GB300 (sm_103a) implementation of the USP-FPM particle update.

The compute path lives in the CUDA library ``libusp.so`` (``csrc/``) behind the
C ABI declared in ``include/usp.h``; ``usp`` is its thin ctypes binding.
"""
