// Fused x pass, float, P = 12 x 16.
#include "kernels_xfused.cuh"
NS3D_XFUSED_VARIANT(float, 12, 16)
