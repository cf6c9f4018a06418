// Kernel instantiations for periodic boundary conditions, grid of 192 points
// per axis (template argument: half the grid).
#include "exx_ops.cuh"
EXX_DEFINE_OPS_PER(96)
