// Kernel instantiations of the exact-exchange pipeline for n = 10 12 14 16 18 20,
// and wire boundary conditions for n = 16.
#include "exx_ops.cuh"
EXX_DEFINE_OPS(10)
EXX_DEFINE_OPS(12)
EXX_DEFINE_OPS(14)
EXX_DEFINE_OPS(16)
EXX_DEFINE_OPS(18)
EXX_DEFINE_OPS(20)
EXX_DEFINE_OPS_WIRE(16)
