// Kernel instantiations of the exact-exchange pipeline for n = 96,
// and wire boundary conditions for n = 96.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(96)
EXX_DEFINE_OPS_WIRE(96)
