// Column pass: float, sign -1, first pass column-fast=false, last pass column-fast=true.
#include "kernels_col.cuh"
NS3D_COL_VARIANT(float, -1, false, true)
