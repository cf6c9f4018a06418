// Kernel instantiations of the exact-exchange pipeline for n = 112.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(112)
