// Kernel instantiations for periodic boundary conditions, grids of 8 .. 64
// points per axis (template argument: half the grid).
#include "exx_ops.cuh"
EXX_DEFINE_OPS_PER(4)
EXX_DEFINE_OPS_PER(6)
EXX_DEFINE_OPS_PER(8)
EXX_DEFINE_OPS_PER(12)
EXX_DEFINE_OPS_PER(16)
EXX_DEFINE_OPS_PER(24)
EXX_DEFINE_OPS_PER(32)
