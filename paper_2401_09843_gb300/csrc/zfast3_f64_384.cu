// Three-pass register z pass, double, P = 8 x 8 x 6.
#include "kernels_long.cuh"
NS3D_ZFAST3_VARIANT(double, 8, 8, 6)
