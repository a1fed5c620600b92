// Fused z pass, double.
#include "kernels_z.cuh"
NS3D_Z_VARIANT(double)
