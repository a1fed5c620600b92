// Register-resident column pass (colfast_f32_*.cu): one kernel per (sign, N1, N2).
#pragma once

#include "kernels_col.cuh"
#include "ns3d_colfast.cuh"

namespace ns3d {

template <typename T, int SIGN, int N1, int N2>
__global__ void __launch_bounds__(ColFastShape<N1, N2>::NTHR, ColFastShape<N1, N2>::MINB)
    k_colfast(ColArgs<T> a) {
  using S = ColFastShape<N1, N2>;
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(ns3d_smem);
  cplx<T>* X = tw + S::P;
  colfast_twiddles<T, SIGN, N1, N2>(tw, a.tw, threadIdx.x, S::NTHR);
  __syncthreads();
  colfast_pass1<T, SIGN, N1, N2, (SIGN > 0)>(a, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, S::NTHR, tw, X);
  __syncthreads();
  colfast_pass2<T, SIGN, N1, N2, (SIGN < 0)>(a, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, S::NTHR, X);
}

template <typename T, int SIGN, int N1, int N2>
cudaError_t colfast_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s) {
  using S = ColFastShape<N1, N2>;
  const size_t smem = (size_t)S::SM_ELEMS * sizeof(cplx<T>);
  dim3 grid((a.ncols + S::W - 1) / S::W, L.gy, L.gz);
  k_colfast<T, SIGN, N1, N2><<<grid, S::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int SIGN, int N1, int N2>
cudaError_t colfast_init() {
  return cudaFuncSetAttribute((const void*)k_colfast<T, SIGN, N1, N2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace ns3d

#define NS3D_COLFAST_VARIANT(T, N1, N2)                                                       \
  namespace ns3d {                                                                           \
  template cudaError_t colfast_launch<T, +1, N1, N2>(const ColArgs<T>&, const Launch&,        \
                                                     cudaStream_t);                           \
  template cudaError_t colfast_launch<T, -1, N1, N2>(const ColArgs<T>&, const Launch&,        \
                                                     cudaStream_t);                           \
  template cudaError_t colfast_init<T, +1, N1, N2>();                                        \
  template cudaError_t colfast_init<T, -1, N1, N2>();                                        \
  }
