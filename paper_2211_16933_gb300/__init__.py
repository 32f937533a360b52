"""GB300 (sm_103a) solver for the finite-difference Enskog-Shakhov lattice Boltzmann
model of arXiv:2211.16933.  The compute path is the CUDA library libqlbm.so
(C ABI in include/qlbm.h); ``qlbm`` is its thin Python binding."""
