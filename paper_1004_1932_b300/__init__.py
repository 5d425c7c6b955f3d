"""B300-native active-dumbbell suspension library.

``inputs`` draws seeded initial conditions; ``dbs`` is the ctypes binding of
the C-ABI library ``libdbs.so`` (CUDA, sm_103a).  Importing the package does
not load the CUDA library; ``dbs.load()`` does, and fails loudly when the
library is missing.
"""
__all__ = ["inputs"]
