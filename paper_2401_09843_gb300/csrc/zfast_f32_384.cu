// Register-resident z pass, float, P = 24 x 16.
#include "kernels_zfast.cuh"
NS3D_ZFAST_VARIANT(float, 24, 16)
