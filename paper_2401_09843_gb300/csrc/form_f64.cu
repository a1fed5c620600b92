// Nonlinear forms 1 and 2, double.
#include "kernels_form.cuh"
NS3D_FORM_VARIANT(double)
