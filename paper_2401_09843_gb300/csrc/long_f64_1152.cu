// Three-pass register z pass, double, P = 16 x 9 x 8.
#include "kernels_long.cuh"
NS3D_ZFAST3_VARIANT(double, 16, 9, 8)
