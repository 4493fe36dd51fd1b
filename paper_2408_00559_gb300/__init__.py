"""GB300 (sm_103a) implementation of the AMFR-W2 sparse-grid solver for the
SABR-LMM pricing PDE (arXiv 2408.00559).

The compute path is the CUDA library ``libamfrw.so`` (C ABI in
``include/amfrw.h``); ``_lib`` is its ctypes binding.  ``workloads`` draws the
seeded synthetic inputs.  Importing this package does not load the library;
the first call into the binding does, and fails loudly if it is missing.
"""
from . import workloads  # noqa: F401
from ._lib import Batch, Problem, solve_batch  # noqa: F401
