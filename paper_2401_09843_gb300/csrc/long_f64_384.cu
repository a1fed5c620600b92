// Three-pass register column passes, double, P = 16 x 4 x 6 (the z pass at
// this size is 8 x 8 x 6, zfast3_f64_384.cu).
#include "kernels_long.cuh"
NS3D_COLFAST3_VARIANT(double, 16, 4, 6)
