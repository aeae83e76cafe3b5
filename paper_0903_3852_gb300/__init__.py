"""GB300-native ensemble integration of stochastic differential equations.

Hot path of Januszewski & Kostur (arXiv:0903.3852): many independent SDE paths
advanced by the SRK2 step of Alg. 2 with counter-based Gaussian noise, for the
driven Josephson-junction phase equation (Eq. 1) and the noisy Kuramoto model
(Eq. 2), with on-device FP64 ensemble reductions.  The compute runs in the CUDA
library built from csrc/ (C ABI declared in include/sde.h); the Python binding
in ``sde`` only marshals arguments.  Importing this package does not load the
library; ``sde.lib()`` does, and raises if it is missing.
"""
