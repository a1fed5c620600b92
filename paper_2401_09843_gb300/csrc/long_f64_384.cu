// Three-pass register kernels, double, P = 16 x 4 x 6.
#include "kernels_long.cuh"
NS3D_LONG_VARIANT(double, 16, 4, 6)
