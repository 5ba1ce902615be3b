"""GB300-native particle-mesh kick with linear-response massive neutrinos.

The compute path is the C-ABI library ``libnupm`` (hand-written CUDA for
sm_103a) declared in ``include/nupm.h``; ``paper_1209_0461_gb300.nupm`` is its
thin ctypes binding.  ``synth`` generates seeded synthetic inputs.  Importing
the package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
__all__ = ["nupm", "synth"]
