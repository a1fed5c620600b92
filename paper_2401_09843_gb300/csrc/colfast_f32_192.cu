// Register-resident column pass, float, P = 12 x 16.
#include "kernels_colfast.cuh"
NS3D_COLFAST_VARIANT(float, 12, 16)
