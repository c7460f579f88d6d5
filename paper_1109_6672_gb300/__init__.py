"""GB300-native coupled DDF thermal lattice Boltzmann (D2Q9) after
Li, Luo, He, Gao & Tao, arXiv:1109.6672.

The compute path is the CUDA library ``liblbm.so`` (built from ``csrc/``) behind
the C-ABI declared in ``include/lbm.h``; ``paper_1109_6672_gb300.lbm`` is its
ctypes binding.  ``inputs`` holds the seeded synthetic workloads.
"""
