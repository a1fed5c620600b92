// Fused x pass kernels (xfused_f32_*.cu): one kernel per (N1, N2).
//
// One CTA per W (ky, kz) columns of one member.  Thread 0 keeps the staging
// ring full with TMA tile loads (tile j into slot j % NSLOT, issued once tile
// j - NSLOT has been read by every thread); each slot has an mbarrier whose
// phase parity is (j / NSLOT) & 1.  A wait that times out sets the member's
// TIMEOUT flag; the CTA then drains its outstanding copies (bounded) and
// returns.
#pragma once

#include "kernels_col.cuh"
#include "ns3d_tma.cuh"
#include "ns3d_xfused.cuh"

namespace ns3d {

// blocks per SM the registers are capped for: 12 warps, or 18 at P = 96 (96
// registers; 149 uncapped allowed four blocks of three warps)
template <int N1, int N2>
constexpr int xfused_minb() {
  return (N1 == 12 && N2 == 8) ? 6
                               : (XFusedShape<N1, N2>::NTHR <= 192 ? 384 / XFusedShape<N1, N2>::NTHR : 1);
}

template <typename T, int N1, int N2>
__global__ void __launch_bounds__(XFusedShape<N1, N2>::NTHR, xfused_minb<N1, N2>())
    k_xfused(const XFusedArgs<T> a, const __grid_constant__ XFusedMaps maps) {
  using S = XFusedShape<N1, N2>;
  extern __shared__ __align__(128) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  cplx<T>* ring = sm;
  cplx<T>* tw = sm + S::OFF_TW;
  cplx<T>* X = sm + S::OFF_X;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + S::SM_ELEMS);
  const int tid = threadIdx.x, bx = blockIdx.x, m = blockIdx.y;
  const int L = xf_num_tiles(a.stage);
  constexpr uint32_t kTileBytes = S::SLOT * sizeof(cplx<T>);

  auto issue = [&](int j) {
    const XfTile t = xf_tile<N1, N2>(j, m, a.stage);
    const CUtensorMap* mp = t.src == 0 ? &maps.dq : (t.src == 1 ? &maps.u0 : &maps.us);
    uint64_t* b = bar + j % S::NSLOT;
    mbar_arrive_expect_tx(b, j == 0 ? kTileBytes + a.extra_tx : kTileBytes);
    tma_load_2d(ring + (j % S::NSLOT) * S::SLOT, mp, 2 * bx * S::W, (int)t.row, b);
  };

  if (tid == 0) {
    for (int i = 0; i < S::NSLOT; ++i) mbar_init(bar + i, 1);
    mbar_init_fence();
    for (int j = 0; j < S::NSLOT && j < L; ++j) issue(j);
  }
  int issued = S::NSLOT < L ? S::NSLOT : L;
  xfused_twiddles<T, N1, N2>(a, tw, tid, S::NTHR);
  XFusedState<T, N1, N2> st;
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int k = 0; k < N2; ++k) st.v[q][k] = czero<T>();
  __syncthreads();

  bool fail = false;
  // forward transforms of the six product components
#pragma unroll 1
  for (int q = 0; q < 6; ++q) {
    for (int j = 3 * q; j < 3 * q + 3; ++j)
      fail |= !mbar_wait(bar + j % S::NSLOT, (j / S::NSLOT) & 1);
    xfused_fwd1<T, N1, N2>(q, tid, S::NTHR, ring, tw, X);
    if (__syncthreads_or(fail)) goto bail;
    if (tid == 0) {
      fence_async_smem();
      for (int j = 3 * q + S::NSLOT; j < 3 * q + 3 + S::NSLOT && j < L; ++j) issue(j);
    }
    issued = min(L, 3 * q + 3 + S::NSLOT);
    xfused_fwd2<T, N1, N2>(a, bx, q, tid, X, st);
    __syncthreads();
  }
  xfused_leray<T, N1, N2>(a, bx, tid, st);
  // per state component: RK3 combine, store, inverse transform
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    const int cl = xf_comp_tiles(a.stage), j0 = 18 + q * cl;
    for (int j = j0; j < j0 + cl; ++j) fail |= !mbar_wait(bar + j % S::NSLOT, (j / S::NSLOT) & 1);
    if (__syncthreads_or(fail)) goto bail;
    {
      cplx<T> v[N2];
      xfused_combine<T, N1, N2>(a, bx, m, q, tid, ring, st, v);
      xfused_inv1<T, N1, N2>(tid, tw, X, v);
    }
    __syncthreads();
    if (tid == 0) {
      fence_async_smem();
      for (int j = j0 + S::NSLOT; j < j0 + cl + S::NSLOT && j < L; ++j) issue(j);
    }
    issued = min(L, j0 + cl + S::NSLOT);
    xfused_inv2<T, N1, N2>(a, bx, m, q, tid, S::NTHR, X);
    __syncthreads();
  }
  xfused_clock<T, N1, N2>(a, bx, m, tid);
  return;

bail:
  // a tile never arrived: flag the member, let the copies still in flight
  // (at most the last NSLOT issued) land before the CTA's memory is released
  if (tid == 0) {
    atomicOr(&a.ctrl[m].status, NS3D_FLAG_TIMEOUT);
    for (int j = issued > S::NSLOT ? issued - S::NSLOT : 0; j < issued; ++j)
      mbar_wait(bar + j % S::NSLOT, (j / S::NSLOT) & 1, 100000000ull);
  }
}

// x-inverse of the stored state with the fused pass's own inverse phases
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(XFusedShape<N1, N2>::NTHR)
    k_xfused_prologue(const XFusedArgs<T> a) {
  using S = XFusedShape<N1, N2>;
  extern __shared__ __align__(128) unsigned char ns3d_smem[];
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(ns3d_smem);
  cplx<T>* X = tw + 2 * S::P;
  const int tid = threadIdx.x, bx = blockIdx.x, m = blockIdx.y;
  xfused_twiddles<T, N1, N2>(a, tw, tid, S::NTHR);
  __syncthreads();
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    {
      cplx<T> v[N2];
      xfused_prologue_load<T, N1, N2>(a, bx, m, q, tid, v);
      xfused_inv1<T, N1, N2>(tid, tw, X, v);
    }
    __syncthreads();
    xfused_inv2<T, N1, N2>(a, bx, m, q, tid, S::NTHR, X);
    __syncthreads();
  }
}

template <typename T, int N1, int N2>
constexpr size_t xfused_prologue_smem() {
  using S = XFusedShape<N1, N2>;
  return (size_t)(2 * S::P + S::W * S::LP) * sizeof(cplx<T>);
}

template <typename T, int N1, int N2>
cudaError_t xfused_prologue_launch(const XFusedArgs<T>& a, int nm, cudaStream_t s) {
  using S = XFusedShape<N1, N2>;
  const int ncols = a.N * a.h;
  if (ncols % S::W != 0 || 2 * S::H != a.N) return cudaErrorInvalidValue;
  k_xfused_prologue<T, N1, N2><<<dim3(ncols / S::W, nm), S::NTHR, xfused_prologue_smem<T, N1, N2>(), s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
constexpr size_t xfused_smem_bytes() {
  using S = XFusedShape<N1, N2>;
  return (size_t)S::SM_ELEMS * sizeof(cplx<T>) + S::NSLOT * sizeof(uint64_t);
}

template <typename T, int N1, int N2>
cudaError_t xfused_launch(const XFusedArgs<T>& a, const XFusedMaps& maps, int nm, cudaStream_t s) {
  using S = XFusedShape<N1, N2>;
  const int ncols = a.N * a.h;
  if (ncols % S::W != 0 || 2 * S::H != a.N) return cudaErrorInvalidValue;
  dim3 grid(ncols / S::W, nm);
  k_xfused<T, N1, N2><<<grid, S::NTHR, xfused_smem_bytes<T, N1, N2>(), s>>>(a, maps);
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
cudaError_t xfused_init() {
  static_assert(xfused_smem_bytes<T, N1, N2>() <= 227 * 1024, "fused x pass: shared memory");
  cudaError_t e = cudaFuncSetAttribute((const void*)k_xfused<T, N1, N2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)xfused_smem_bytes<T, N1, N2>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute((const void*)k_xfused_prologue<T, N1, N2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)xfused_prologue_smem<T, N1, N2>());
}

}  // namespace ns3d

#define NS3D_XFUSED_VARIANT(T, N1, N2)                                                      \
  namespace ns3d {                                                                         \
  template cudaError_t xfused_launch<T, N1, N2>(const XFusedArgs<T>&, const XFusedMaps&, int, \
                                                cudaStream_t);                             \
  template cudaError_t xfused_init<T, N1, N2>();                                           \
  template cudaError_t xfused_prologue_launch<T, N1, N2>(const XFusedArgs<T>&, int, cudaStream_t); \
  }
