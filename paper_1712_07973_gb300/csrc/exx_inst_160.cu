// Kernel instantiations of the exact-exchange pipeline for n = 160.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(160)
