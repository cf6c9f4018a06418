// Kernel instantiations for periodic boundary conditions, grids of 96 and 128
// points per axis, and slab boundary conditions on the grid of 96 (template
// argument: half the grid).
#include "exx_ops.cuh"
EXX_DEFINE_OPS_PER(48)
EXX_DEFINE_OPS_PER(64)
EXX_DEFINE_OPS_SLAB(48)
