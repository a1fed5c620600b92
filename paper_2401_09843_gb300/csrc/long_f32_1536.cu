// Three-pass register kernels, float, P = 16 x 12 x 8.
#include "kernels_long.cuh"
NS3D_LONG_VARIANT(float, 16, 12, 8)
