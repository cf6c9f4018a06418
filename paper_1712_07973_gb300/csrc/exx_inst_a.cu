// Kernel instantiations of the exact-exchange pipeline for n = 2 3 4 5 6 7 8 9,
// and wire boundary conditions for n = 8 (x and y transforms as for free ones).
#include "exx_ops.cuh"
EXX_DEFINE_OPS(2)
EXX_DEFINE_OPS(3)
EXX_DEFINE_OPS(4)
EXX_DEFINE_OPS(5)
EXX_DEFINE_OPS(6)
EXX_DEFINE_OPS(7)
EXX_DEFINE_OPS(8)
EXX_DEFINE_OPS(9)
EXX_DEFINE_OPS_WIRE(8)
