"""B300-native D2Q37 thermal lattice Boltzmann step (Ripesi et al., PRE 89, 043022).

The compute path is the CUDA library ``csrc/liblbm.so`` behind the C-ABI declared in
``include/lbm.h``; ``lbm`` is its thin ctypes binding.  Importing this package does not
load the library; ``paper_1405_1253_b300.lbm`` does, and fails loudly if it is missing.
"""
__all__ = ["workloads"]
