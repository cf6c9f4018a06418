// Kernel instantiations of the exact-exchange pipeline for n = 24 28 32 36 40.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(24)
EXX_DEFINE_OPS(28)
EXX_DEFINE_OPS(32)
EXX_DEFINE_OPS(36)
EXX_DEFINE_OPS(40)
