"""GB300-native PASD (Parallel Active Subspace Decomposition) solver for tensor RPCA.

The solver itself is the C-ABI library ``libpasd.so`` (CUDA, sm_103a); ``pasd``
is its thin ctypes binding. Importing this package does not load the library;
``from paper_1712_09999_gb300 import pasd`` does, and fails loudly if it has not
been built.
"""
