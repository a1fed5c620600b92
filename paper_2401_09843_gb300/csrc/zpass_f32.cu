// Fused z pass, float.
#include "kernels_z.cuh"
NS3D_Z_VARIANT(float)
