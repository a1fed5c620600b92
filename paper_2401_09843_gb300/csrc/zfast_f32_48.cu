// Register-resident z pass, float, P = 6 x 8.
#include "kernels_zfast.cuh"
NS3D_ZFAST_VARIANT(float, 6, 8)
