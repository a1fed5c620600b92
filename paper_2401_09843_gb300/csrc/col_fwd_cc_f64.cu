// Column pass: double, sign -1, first pass column-fast=true, last pass column-fast=true.
#include "kernels_col.cuh"
NS3D_COL_VARIANT(double, -1, true, true)
