// Kernel instantiations for periodic boundary conditions, grids of 8 .. 64
// points per axis, and slab boundary conditions on grids of 8 .. 64 (their x
// and y transforms are the periodic ones; template argument: half the grid).
#include "exx_ops.cuh"
EXX_DEFINE_OPS_PER(4)
EXX_DEFINE_OPS_PER(6)
EXX_DEFINE_OPS_PER(8)
EXX_DEFINE_OPS_PER(12)
EXX_DEFINE_OPS_PER(16)
EXX_DEFINE_OPS_PER(24)
EXX_DEFINE_OPS_PER(32)
EXX_DEFINE_OPS_SLAB(4)
EXX_DEFINE_OPS_SLAB(8)
EXX_DEFINE_OPS_SLAB(16)
EXX_DEFINE_OPS_SLAB(24)
EXX_DEFINE_OPS_SLAB(32)
