// Point-wise kernels, float.
#include "kernels_misc.cuh"
NS3D_MISC_VARIANT(float)
