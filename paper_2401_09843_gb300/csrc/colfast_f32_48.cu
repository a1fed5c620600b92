// Register-resident column pass, float, P = 6 x 8.
#include "kernels_colfast.cuh"
NS3D_COLFAST_VARIANT(float, 6, 8)
