// Column-pass kernel (one variant per translation unit, see col_*.cu).
#pragma once

#include "ns3d_launch.h"

namespace ns3d {

struct DevSync {
  NS3D_HD void operator()() const {
#if defined(__CUDA_ARCH__)
    __syncthreads();
#endif
  }
};

template <typename T, int SIGN, bool CF1, bool CFL>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 256) k_col(ColArgs<T> a) {
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  colfft_block<T, SIGN, CF1, CFL>(a, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, blockDim.x,
                                  reinterpret_cast<cplx<T>*>(ns3d_smem), DevSync{});
}

template <typename T, int SIGN, bool CF1, bool CFL>
cudaError_t col_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s) {
  k_col<T, SIGN, CF1, CFL><<<dim3(L.gx, L.gy, L.gz), L.nthr, L.smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int SIGN, bool CF1, bool CFL>
cudaError_t col_init() {
  return cudaFuncSetAttribute((const void*)k_col<T, SIGN, CF1, CFL>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace ns3d

#define NS3D_COL_VARIANT(T, SIGN, CF1, CFL)                                                    \
  namespace ns3d {                                                                             \
  template cudaError_t col_launch<T, SIGN, CF1, CFL>(const ColArgs<T>&, const Launch&,         \
                                                     cudaStream_t);                            \
  template cudaError_t col_init<T, SIGN, CF1, CFL>();                                          \
  }
