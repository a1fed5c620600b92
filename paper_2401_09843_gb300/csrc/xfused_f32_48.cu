// Fused x pass, float, P = 6 x 8.
#include "kernels_xfused.cuh"
NS3D_XFUSED_VARIANT(float, 6, 8)
