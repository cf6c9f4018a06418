// Kernel instantiations of the exact-exchange pipeline for n = 48 56 64,
// and wire boundary conditions for n = 48 and 64.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(48)
EXX_DEFINE_OPS(56)
EXX_DEFINE_OPS(64)
EXX_DEFINE_OPS_WIRE(48)
EXX_DEFINE_OPS_WIRE(64)
