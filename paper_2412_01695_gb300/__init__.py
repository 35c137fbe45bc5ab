"""Many-k Kohn-Sham H|psi>, batched Davidson and DFPT Sternheimer CG on one GB300 (sm_103a).

The compute path is the C-ABI library built from ``csrc/`` (``libpwk.so``); this package
holds its thin ctypes binding (``pwk``), the build step (``build``) and the seeded input
generator (``synth``).  There is no CPU fallback: calls fail loudly if the library or a
CUDA device is missing.
"""
__all__ = ["synth"]
