"""GB300-native hot path of the Palabos Turret time step (arXiv 2408.15115).

The compute lives in ``libturret.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/turret.h``); :mod:`.turret` is a thin ctypes binding that
marshals arguments only.  :mod:`.inputs` makes seeded synthetic shapes and fields.
Importing the package loads nothing; the binding loads the library on first use
and raises if it is missing.
"""
__all__ = ["inputs", "configs", "turret"]
