// Fused z-pass kernel (zpass_f32.cu / zpass_f64.cu).
#pragma once

#include "kernels_col.cuh"

namespace ns3d {

// 512 threads (FP32) when a tile's shared memory allows one block per SM
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 128) k_zfused(ZArgs<T> a) {
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  double* red = reinterpret_cast<double*>(sm + 4 * a.P * a.ldw);
  zfused_block<T>(a, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, blockDim.x, sm, red,
                  DevSync{});
}

template <typename T>
cudaError_t launch_zfused(const ZArgs<T>& a, const Launch& L, cudaStream_t s) {
  k_zfused<T><<<dim3(L.gx, L.gy, L.gz), L.nthr, L.smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t zfused_init() {
  return cudaFuncSetAttribute((const void*)k_zfused<T>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace ns3d

#define NS3D_Z_VARIANT(T)                                                                       \
  namespace ns3d {                                                                             \
  template cudaError_t launch_zfused<T>(const ZArgs<T>&, const Launch&, cudaStream_t);         \
  template cudaError_t zfused_init<T>();                                                       \
  }
