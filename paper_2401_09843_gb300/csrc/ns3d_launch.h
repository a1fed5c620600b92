// Launchers of the solver's kernels.  Each kernel variant lives in its own
// translation unit (col_*.cu, zpass_*.cu, misc_*.cu) so the build compiles
// them in parallel; this header only declares them.
#pragma once

#include <cuda_runtime.h>

#include "ns3d_geom.h"

namespace ns3d {

// Column-pass variants: transform direction and the thread mapping of the
// first / last pass (column-fast when the global data is contiguous across
// columns, task-fast when it is contiguous along the transform axis).
enum ColKind {
  COL_INV_CC = 0,   // inverse, contiguous columns in and out (inverse x)
  COL_INV_CT = 1,   // inverse, columns in, transposed out (inverse y)
  COL_FWD_TC = 2,   // forward, transposed in, columns out (forward y)
  COL_FWD_CC = 3,   // forward, columns in and out (forward x)
};

template <typename T, int SIGN, bool CF1, bool CFL>
cudaError_t col_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s);
template <typename T, int SIGN, bool CF1, bool CFL>
cudaError_t col_init();

template <typename T>
cudaError_t launch_col(const ColArgs<T>& a, ColKind kind, const Launch& L, cudaStream_t s) {
  switch (kind) {
    case COL_INV_CC: return col_launch<T, +1, true, true>(a, L, s);
    case COL_INV_CT: return col_launch<T, +1, true, false>(a, L, s);
    case COL_FWD_TC: return col_launch<T, -1, false, true>(a, L, s);
    case COL_FWD_CC: return col_launch<T, -1, true, true>(a, L, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_zfused(const ZArgs<T>& a, const Launch& L, cudaStream_t s);
template <typename T>
cudaError_t zfused_init();
template <typename T>
cudaError_t launch_spectral(const SpecArgs<T>& a, long long total, cudaStream_t s);
template <typename T>
cudaError_t launch_d1_to_compact(const cplx<T>* d1, cplx<T>* u, int N, cudaStream_t s);
template <typename T>
cudaError_t launch_compact_to_d1(const cplx<T>* u, cplx<T>* d1, int N, cudaStream_t s);

template <typename T>
cudaError_t kernels_init() {
  cudaError_t e[5] = {col_init<T, +1, true, true>(), col_init<T, +1, true, false>(),
                      col_init<T, -1, false, true>(), col_init<T, -1, true, true>(),
                      zfused_init<T>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

cudaError_t launch_ctrl_reset(Ns3dCtrl* c, int n, cudaStream_t s);
cudaError_t launch_ctrl_set_tend(Ns3dCtrl* c, int n, double t_end, cudaStream_t s);

}  // namespace ns3d
