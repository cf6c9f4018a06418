// Kernel instantiations of the exact-exchange pipeline for n = 96.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(96)
