// Kernel instantiations of the exact-exchange pipeline for n = 72 80.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(72)
EXX_DEFINE_OPS(80)
