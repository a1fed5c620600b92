// Three-pass register kernels, float, P = 1536: column passes 16 x 12 x 8,
// z pass 24 x 8 x 8.
#include "kernels_long.cuh"
NS3D_COLFAST3_VARIANT(float, 16, 12, 8)
NS3D_ZFAST3_VARIANT(float, 24, 8, 8)
