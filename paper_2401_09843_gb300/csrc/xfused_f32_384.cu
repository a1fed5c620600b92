// Fused x pass, float, P = 24 x 16.
#include "kernels_xfused.cuh"
NS3D_XFUSED_VARIANT(float, 24, 16)
