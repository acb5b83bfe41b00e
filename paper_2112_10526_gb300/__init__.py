"""GB300-native RBM variational Monte Carlo hot path (NetKet 3, arXiv:2112.10526).

The compute path is the C-ABI library ``libnk.so`` (hand-written sm_103a
CUDA) declared in ``include/nk.h``; ``paper_2112_10526_gb300.nk`` is its thin
ctypes binding.  Importing this package does not load the library; the first
call into ``nk`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "nk"]
