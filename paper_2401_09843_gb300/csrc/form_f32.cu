// Nonlinear forms 1 and 2, float.
#include "kernels_form.cuh"
NS3D_FORM_VARIANT(float)
