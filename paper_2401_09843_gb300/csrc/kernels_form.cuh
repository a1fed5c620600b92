// Forms 1 and 2 of the nonlinear term (form_f32.cu / form_f64.cu): the
// spectral fields of the form and the z pass that forms the products.
#pragma once

#include "kernels_col.cuh"

namespace ns3d {

// grid.y = member; threads stride over the member's N N h modes
template <typename T>
__global__ void k_form_prep(const cplx<T>* u, cplx<T>* F, int N, T kscale, int form,
                            long long mu, long long mf) {
  const long long plane = (long long)N * N * (N / 2);
  const cplx<T>* um = u + blockIdx.y * mu;
  cplx<T>* Fm = F + blockIdx.y * mf;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x)
    form_prep_point<T>(um, Fm, N, kscale, form, i);
}

template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 512 : 128) k_zform(ZArgs<T> a, int form) {
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  double* red = reinterpret_cast<double*>(sm + (long long)zform_buffers(form) * a.P * a.ldw);
  zform_block<T>(a, form, blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, blockDim.x, sm, red,
                 DevSync{});
}

template <typename T>
cudaError_t launch_form_prep(const cplx<T>* u, cplx<T>* F, int N, T kscale, int form, long long mu,
                             long long mf, int nm, cudaStream_t s) {
  const long long plane = (long long)N * N * (N / 2);
  long long gx = (plane + 255) / 256;
  if (gx > 152LL * 8) gx = 152LL * 8;
  k_form_prep<T><<<dim3((unsigned)gx, nm), 256, 0, s>>>(u, F, N, kscale, form, mu, mf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zform(const ZArgs<T>& a, int form, const Launch& L, cudaStream_t s) {
  k_zform<T><<<dim3(L.gx, L.gy, L.gz), L.nthr, L.smem, s>>>(a, form);
  return cudaGetLastError();
}

template <typename T>
cudaError_t zform_init() {
  return cudaFuncSetAttribute((const void*)k_zform<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024);
}

}  // namespace ns3d

#define NS3D_FORM_VARIANT(T)                                                                     \
  namespace ns3d {                                                                              \
  template cudaError_t launch_form_prep<T>(const cplx<T>*, cplx<T>*, int, T, int, long long,    \
                                           long long, int, cudaStream_t);                       \
  template cudaError_t launch_zform<T>(const ZArgs<T>&, int, const Launch&, cudaStream_t);      \
  template cudaError_t zform_init<T>();                                                         \
  }
