"""mfs: matrix-free first-order conic solver (arXiv 2203.05027) for NVIDIA B300 (sm_103a).

The solver itself is the C-ABI library ``libmfs.so`` built from ``csrc/`` (CUDA kernels for the
per-iteration sweep over A's nonzeros, the cone projections and the FP64 residual reductions).
``mfs`` is a thin ctypes binding to it; ``instances`` holds the seeded problem generators.
Importing this package does not load the CUDA library; ``mfs.load()`` does, and fails loudly if
it is missing.
"""
