"""GB300-native decoupled Hermite-expansion lattice Boltzmann solver.

The compute path is a CUDA C-ABI library (``liblbm.so``, built for sm_103a
from ``csrc/``) that advances the translational and rotational populations of
Hu, Zhang & Geng's decoupled scheme (arXiv 1606.06107).  ``lbm`` is a thin
ctypes binding over it; PyTorch supplies only device memory and streams.
"""
from .lbm import Lbm, LbmBatch, LbmError, load_library  # noqa: F401
