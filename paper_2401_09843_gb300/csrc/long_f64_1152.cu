// Three-pass register kernels, double, P = 16 x 9 x 8.
#include "kernels_long.cuh"
NS3D_LONG_VARIANT(double, 16, 9, 8)
