// Register-resident z pass, float, P = 12 x 16.
#include "kernels_zfast.cuh"
NS3D_ZFAST_VARIANT(float, 12, 16)
