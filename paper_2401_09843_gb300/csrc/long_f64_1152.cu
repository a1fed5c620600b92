// Three-pass register kernels, double, P = 1152: column passes 16 x 9 x 8,
// z pass 12 x 12 x 8.
#include "kernels_long.cuh"
NS3D_COLFAST3_VARIANT(double, 16, 9, 8)
NS3D_ZFAST3_VARIANT(double, 12, 12, 8)
