"""GB300-native energy-parallel NEGF / recursive Green's function library.

The compute path is the C-ABI shared library ``libnegf.so`` built from ``csrc/`` (CUDA for
sm_103a); ``negf`` is its thin ctypes binding.  Importing this package does not load the
library; ``paper_2407_14633_gb300.negf.load()`` does, and raises if it is missing.
"""
__all__ = ["negf", "synth"]
