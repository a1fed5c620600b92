// Three-pass register kernels for long lines (long_f32_*.cu): column pass
// and fused z pass, one instantiation per (N1, N2, N3).
#pragma once

#include "kernels_col.cuh"
#include "ns3d_colfast3.cuh"
#include "ns3d_zfast3.cuh"

namespace ns3d {

template <typename T, int SIGN, int N1, int N2, int N3>
__global__ void __launch_bounds__(ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>::NTHR) k_colfast3(ColArgs<T> a) {
  using S = ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>;
  static_assert(sizeof(cplx<LongC<T>>) == sizeof(cplx<T>), "arithmetic and storage types of one size");
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<LongC<T>>* tw = reinterpret_cast<cplx<LongC<T>>*>(ns3d_smem);
  cplx<LongC<T>>* X = tw + S::P;
  const int tid = threadIdx.x;
  colfast3_twiddles<T, SIGN, S::P>(tw, a.tw, tid, S::NTHR);
  __syncthreads();
  colfast3_pass1<T, SIGN, N1, N2, N3, (SIGN > 0)>(a, blockIdx.x, blockIdx.y, blockIdx.z, tid,
                                                  S::NTHR, tw, X);
  __syncthreads();
  const int ncol = imin(S::W, a.ncols - (int)blockIdx.x * S::W);
  colfast3_pass2<T, SIGN, N1, N2, N3>(tid, S::NTHR, ncol, tw, X);
  __syncthreads();
  colfast3_pass3<T, SIGN, N1, N2, N3, (SIGN < 0)>(a, blockIdx.x, blockIdx.y, blockIdx.z, tid,
                                                  S::NTHR, X);
}

template <typename T, int SIGN, int N1, int N2, int N3>
cudaError_t colfast3_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s) {
  using S = ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>;
  const size_t smem = (size_t)S::SM_ELEMS * sizeof(cplx<T>);
  dim3 grid((a.ncols + S::W - 1) / S::W, L.gy, L.gz);
  k_colfast3<T, SIGN, N1, N2, N3><<<grid, S::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N1, int N2, int N3>
__global__ void __launch_bounds__(ZFast3Shape<N1, N2, N3>::NTHR,
                                  sizeof(T) == 8 ? (ZFast3Shape<N1, N2, N3>::NTHR >= 128 ? 2 : 4) : 3)
    k_zfast3(ZArgs<T> a, long long ntiles) {
  using S = ZFast3Shape<N1, N2, N3>;
  using C = LongC<T>;
  static_assert(sizeof(cplx<C>) == sizeof(cplx<T>), "arithmetic and storage types of one size");
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<C>* sm = reinterpret_cast<cplx<C>*>(ns3d_smem);
  T* red = reinterpret_cast<T*>(sm + S::SM_ELEMS);
  const int tid = threadIdx.x;
  zfast3_twiddles<T, N1, N2, N3>(a, sm, tid, S::NTHR);
  ZFast3State<T, N1, N2, N3> st;
  st.umax = C(0);
  st.chk = C(0);
  int cur = -1;
  __syncthreads();
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int bz, by, y0;
    zfast3_tile<N1, N2, N3>(t, &bz, &by, &y0);
    if (bz != cur) {                       // uniform over the block
      if (cur >= 0 && a.ctrl) {
        red[tid] = zfast3_red_value(st);
        __syncthreads();
        if (tid < 32) zfast3_flush<T>(a, cur, red, S::NTHR, tid);
        __syncthreads();
      }
      st.umax = C(0);
      st.chk = C(0);
      cur = bz;
    }
    const ZFast3Ctx<T, N1, N2, N3> c = zfast3_ctx<T, N1, N2, N3>(a, bz, by, y0, sm);
    zfast3_inv1(c, tid, S::NTHR);
    __syncthreads();
    zfast3_inv2(c, tid, S::NTHR);
    __syncthreads();
    zfast3_inv3(c, tid, st);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      zfast3_fwdA(c, tid, st, r);
      __syncthreads();
      zfast3_fwdB(c, tid, S::NTHR);
      __syncthreads();
      zfast3_fwdC(c, tid, S::NTHR);
      __syncthreads();
      zfast3_extract(c, tid, S::NTHR, r);
      __syncthreads();
    }
  }
  if (cur >= 0 && a.ctrl) {
    red[tid] = zfast3_red_value(st);
    __syncthreads();
    if (tid < 32) zfast3_flush<T>(a, cur, red, S::NTHR, tid);
  }
}

template <typename T, int N1, int N2, int N3>
constexpr size_t zfast3_smem() {
  using S = ZFast3Shape<N1, N2, N3>;
  return (size_t)S::SM_ELEMS * sizeof(cplx<T>) + (size_t)S::NTHR * sizeof(T);
}

template <typename T, int N1, int N2, int N3>
cudaError_t zfast3_launch(const ZArgs<T>& a, int nm, cudaStream_t s) {
  using S = ZFast3Shape<N1, N2, N3>;
  const long long ntiles = (long long)nm * S::P * (S::P / 2);
  // persistent blocks: as many as are resident at once
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_zfast3<T, N1, N2, N3>, S::NTHR,
                                                    zfast3_smem<T, N1, N2, N3>()) != cudaSuccess)
    return cudaGetLastError();
  const long long grid = std::min<long long>(ntiles, (long long)std::max(per_sm, 1) * nsm);
  k_zfast3<T, N1, N2, N3><<<(unsigned)grid, S::NTHR, zfast3_smem<T, N1, N2, N3>(), s>>>(a, ntiles);
  return cudaGetLastError();
}

template <typename T, int N1, int N2, int N3>
cudaError_t zfast3_init() {
  static_assert(zfast3_smem<T, N1, N2, N3>() <= 227 * 1024, "three-pass z: shared memory");
  return cudaFuncSetAttribute((const void*)k_zfast3<T, N1, N2, N3>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

template <typename T, int N1, int N2, int N3>
cudaError_t long_init() {
  static_assert(ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>::SM_ELEMS * sizeof(cplx<T>) <= 227 * 1024,
                "three-pass column: shared memory");
  const void* f[2] = {(const void*)k_colfast3<T, +1, N1, N2, N3>,
                      (const void*)k_colfast3<T, -1, N1, N2, N3>};
  for (const void* k : f) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ns3d

// the column passes of one factorisation
#define NS3D_COLFAST3_VARIANT(T, N1, N2, N3)                                                  \
  namespace ns3d {                                                                           \
  template cudaError_t colfast3_launch<T, +1, N1, N2, N3>(const ColArgs<T>&, const Launch&,   \
                                                          cudaStream_t);                      \
  template cudaError_t colfast3_launch<T, -1, N1, N2, N3>(const ColArgs<T>&, const Launch&,   \
                                                          cudaStream_t);                      \
  template cudaError_t long_init<T, N1, N2, N3>();                                           \
  }

// the z pass alone
#define NS3D_ZFAST3_VARIANT(T, N1, N2, N3)                                                    \
  namespace ns3d {                                                                           \
  template cudaError_t zfast3_launch<T, N1, N2, N3>(const ZArgs<T>&, int, cudaStream_t);      \
  template cudaError_t zfast3_init<T, N1, N2, N3>();                                         \
  }

// both, where the z pass and the column passes share the factorisation
#define NS3D_LONG_VARIANT(T, N1, N2, N3) \
  NS3D_COLFAST3_VARIANT(T, N1, N2, N3)   \
  NS3D_ZFAST3_VARIANT(T, N1, N2, N3)
