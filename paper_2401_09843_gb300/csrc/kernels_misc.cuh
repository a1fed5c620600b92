// Point-wise kernels: spectral step / RK3 combine and layout conversions
// (misc_f32.cu / misc_f64.cu).
#pragma once

#include "ns3d_launch.h"

namespace ns3d {

static inline int grid_for(long long total, int nthr) {
  long long g = (total + nthr - 1) / nthr;
  if (g > 152LL * 16) g = 152LL * 16;
  return (int)(g < 1 ? 1 : g);
}

// grid.y = member * N + kx; threads stride over the (ky, kz) plane
template <typename T>
__global__ void __launch_bounds__(256) k_spectral(SpecArgs<T> a) {
  const int m = blockIdx.y / a.N, kx = blockIdx.y % a.N;
  const int plane = a.N * a.h;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < plane; j += gridDim.x * blockDim.x)
    spectral_point<T>(a, m, kx, j);
}

// D1 [3][N][N][h+1] -> compact [3][N][N][h] with the Nyquist rows zeroed
template <typename T>
__global__ void k_d1_to_compact(const cplx<T>* d1, cplx<T>* u, int N) {
  const int h = N / 2;
  const long long total = 3LL * N * N * h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i % h);
    const long long r = i / h;          // (c * N + x) * N + y
    const int y = (int)(r % N);
    const int x = (int)((r / N) % N);
    cplx<T> v = d1[r * (h + 1) + z];
    if (x == h || y == h) v = czero<T>();
    u[i] = v;
  }
}

template <typename T>
__global__ void k_compact_to_d1(const cplx<T>* u, cplx<T>* d1, int N) {
  const int h = N / 2;
  const long long total = 3LL * N * N * (h + 1);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i % (h + 1));
    const long long r = i / (h + 1);
    d1[i] = (z < h) ? u[r * h + z] : czero<T>();
  }
}

template <typename T>
cudaError_t launch_spectral(const SpecArgs<T>& a, cudaStream_t s) {
  const int plane = a.N * a.h;
  int gx = (plane + 4 * 256 - 1) / (4 * 256);     // about four points per thread
  if (gx < 1) gx = 1;
  k_spectral<T><<<dim3(gx, a.nmem * a.N), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_d1_to_compact(const cplx<T>* d1, cplx<T>* u, int N, cudaStream_t s) {
  k_d1_to_compact<T><<<grid_for(3LL * N * N * (N / 2), 256), 256, 0, s>>>(d1, u, N);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_compact_to_d1(const cplx<T>* u, cplx<T>* d1, int N, cudaStream_t s) {
  k_compact_to_d1<T><<<grid_for(3LL * N * N * (N / 2 + 1), 256), 256, 0, s>>>(u, d1, N);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zpass(const ZArgs<T>& a, const Geom& g, int nm, cudaStream_t s) {
  if (zfast_available<T>(g.P) && 3 * g.h == g.P) {
#define NS3D_ZF_GO(A, B) \
    if (g.P == (A) * (B)) return zfast_launch<float, A, B>(*reinterpret_cast<const ZArgs<float>*>(&a), nm, s);
    NS3D_FOR_ZFAST(NS3D_ZF_GO)
#undef NS3D_ZF_GO
  }
  if (zfast3_available<T>(g.P) && 3 * g.h == g.P) {
    if (sizeof(T) == 4) {
#define NS3D_ZF3_GO(A, B, C) \
      if (g.P == (A) * (B) * (C)) \
        return zfast3_launch<float, A, B, C>(*reinterpret_cast<const ZArgs<float>*>(&a), nm, s);
      NS3D_FOR_ZFAST3(NS3D_ZF3_GO)
#undef NS3D_ZF3_GO
    } else {
#define NS3D_ZF3D_GO(A, B, C) \
      if (g.P == (A) * (B) * (C)) \
        return zfast3_launch<double, A, B, C>(*reinterpret_cast<const ZArgs<double>*>(&a), nm, s);
      NS3D_FOR_ZFAST3_F64(NS3D_ZF3D_GO)
#undef NS3D_ZF3D_GO
    }
  }
  return launch_zfused<T>(a, ns3d::launch_z(g, nm), s);
}

}  // namespace ns3d

#define NS3D_MISC_VARIANT(T)                                                                    \
  namespace ns3d {                                                                             \
  template cudaError_t launch_spectral<T>(const SpecArgs<T>&, cudaStream_t);                   \
  template cudaError_t launch_d1_to_compact<T>(const cplx<T>*, cplx<T>*, int, cudaStream_t);   \
  template cudaError_t launch_compact_to_d1<T>(const cplx<T>*, cplx<T>*, int, cudaStream_t);   \
  template cudaError_t launch_zpass<T>(const ZArgs<T>&, const Geom&, int, cudaStream_t);      \
  }
