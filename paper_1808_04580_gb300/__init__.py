"""NFFT-based fast summation for graph Laplacians of fully connected
Gaussian-weighted graphs, on one GB300 (sm_103a).

Method: Alfke, Potts, Stoll, Volkmer, "NFFT meets Krylov methods" (2018).
The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/nfl.h``); ``nfl`` is its Python binding.
"""
from .nfl import KERNELS, Batch, NflError, Plan, PRECISIONS, apply_batched, create_batched, fma_rate, library  # noqa: F401
from .autograd import cg_solve  # noqa: F401
