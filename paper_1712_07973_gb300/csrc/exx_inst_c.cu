// Kernel instantiations of the exact-exchange pipeline for n = 24 28 32 36 40,
// and wire boundary conditions for n = 32.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(24)
EXX_DEFINE_OPS(28)
EXX_DEFINE_OPS(32)
EXX_DEFINE_OPS(36)
EXX_DEFINE_OPS(40)
EXX_DEFINE_OPS_WIRE(32)
