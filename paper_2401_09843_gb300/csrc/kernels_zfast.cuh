// Register-resident fused z pass (zfast_f32.cu): one kernel per (N1, N2).
#pragma once

#include "kernels_col.cuh"
#include "ns3d_zfast.cuh"
#include "ns3d_zrot.cuh"
#include "ns3d_zadj.cuh"

namespace ns3d {

template <typename T, int N1, int N2>
// blocks per SM as ZFastShape::MINB (the register-resident state caps residency)
__global__ void __launch_bounds__(ZFastShape<N1, N2>::NTHR, ZFastShape<N1, N2>::MINB) k_zfast(ZArgs<T> a) {
  using S = ZFastShape<N1, N2>;
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  T* red = reinterpret_cast<T*>(sm + S::SM_ELEMS);
  const ZFastCtx<T, N1, N2> c = zfast_ctx<T, N1, N2>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
  const int tid = threadIdx.x;
  zfast_load_twiddles(c, tid, S::NTHR);
  __syncthreads();
  zfast_inv1(c, tid, S::NTHR);
  __syncthreads();
  ZFastState<T, N1, N2> st;
  zfast_inv2(c, tid, st);
  red[tid] = st.bad ? T(-1) : st.umax;
  __syncthreads();
  if (tid < 32) zfast_reduce(c, red, S::NTHR, tid);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    zfast_fwd1(c, tid, st, r);
    __syncthreads();
    zfast_fwd2(c, tid, S::NTHR);
    __syncthreads();
    zfast_extract(c, tid, r);
    __syncthreads();
  }
}

template <typename T, int N1, int N2>
size_t zfast_smem() {
  using S = ZFastShape<N1, N2>;
  return (size_t)S::SM_ELEMS * sizeof(cplx<T>) + (size_t)S::NTHR * sizeof(double);
}

template <typename T, int N1, int N2>
cudaError_t zfast_launch(const ZArgs<T>& a, int nm, cudaStream_t s) {
  using S = ZFastShape<N1, N2>;
  dim3 grid((S::P + S::Y - 1) / S::Y, S::P, nm);
  k_zfast<T, N1, N2><<<grid, S::NTHR, zfast_smem<T, N1, N2>(), s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
cudaError_t zfast_init() {
  return cudaFuncSetAttribute((const void*)k_zfast<T, N1, N2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

// The rotational form's register-resident z pass (ns3d_zrot.cuh), same sizes.
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(ZRotShape<N1, N2>::NTHR, 384 / ZRotShape<N1, N2>::NTHR) k_zrot(ZArgs<T> a) {
  using S = ZRotShape<N1, N2>;
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  T* red = reinterpret_cast<T*>(sm + S::SM_ELEMS);
  const ZFastCtx<T, N1, N2> c = zrot_ctx<T, N1, N2>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
  const int tid = threadIdx.x;
  zfast_load_twiddles(c, tid, S::NTHR);
  __syncthreads();
  zrot_inv1(c, tid, S::NTHR);
  __syncthreads();
  ZFastState<T, N1, N2> st;
  zrot_inv2(c, tid, st);
  red[tid] = st.bad ? T(-1) : st.umax;
  __syncthreads();
  if (tid < 32) zfast_reduce(c, red, S::NTHR, tid);
  zrot_fwd1(c, tid, st);
  __syncthreads();
  zrot_fwd2(c, tid, S::NTHR);
  __syncthreads();
  zrot_extract(c, tid, S::NTHR);
}

template <typename T, int N1, int N2>
size_t zrot_smem() {
  using S = ZRotShape<N1, N2>;
  return (size_t)S::SM_ELEMS * sizeof(cplx<T>) + (size_t)S::NTHR * sizeof(double);
}

template <typename T, int N1, int N2>
cudaError_t zrot_launch(const ZArgs<T>& a, int nm, cudaStream_t s) {
  using S = ZRotShape<N1, N2>;
  dim3 grid((S::P + S::Y - 1) / S::Y, S::P, nm);
  k_zrot<T, N1, N2><<<grid, S::NTHR, zrot_smem<T, N1, N2>(), s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
cudaError_t zrot_init() {
  return cudaFuncSetAttribute((const void*)k_zrot<T, N1, N2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

// The adjoint right-hand side's register-resident z pass (ns3d_zadj.cuh), same sizes.
template <typename T, int N1, int N2>
// (12 warps per SM: four blocks of 96 threads)
__global__ void __launch_bounds__(ZAdjShape<N1, N2>::NTHR, 384 / ZAdjShape<N1, N2>::NTHR) k_zadjf(ZArgs<T> a) {
  using S = ZAdjShape<N1, N2>;
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  const ZFastCtx<T, N1, N2> c = zadjf_ctx<T, N1, N2>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
  const int tid = threadIdx.x;
  zfast_load_twiddles(c, tid, S::NTHR);
  __syncthreads();
  ZAdjState<T, N1, N2> st;
  for (int part = 0; part < 2; ++part) {
    zadjf_inv1(c, tid, S::NTHR, part);
    __syncthreads();
    zadjf_inv2(c, tid, st, part);
    __syncthreads();
  }
  zadjf_fwd1(c, tid, st);
  __syncthreads();
  zadjf_fwd2(c, tid, S::NTHR);
  __syncthreads();
  zadjf_extract(c, tid, S::NTHR);
}

// The advective form's register-resident z pass (ns3d_zadj.cuh, KIND 1), same sizes.
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(ZAdjShape<N1, N2, 1>::NTHR, 384 / ZAdjShape<N1, N2, 1>::NTHR) k_zadv(ZArgs<T> a) {
  using S = ZAdjShape<N1, N2, 1>;
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(ns3d_smem);
  T* red = reinterpret_cast<T*>(sm + S::SM_ELEMS);
  const ZFastCtx<T, N1, N2> c = zadjf_ctx<T, N1, N2, 1>(a, blockIdx.x, blockIdx.y, blockIdx.z, sm);
  const int tid = threadIdx.x;
  zfast_load_twiddles(c, tid, S::NTHR);
  __syncthreads();
  ZAdjState<T, N1, N2> st;
  zadjf_inv1<T, N1, N2, 1>(c, tid, S::NTHR, 0);
  __syncthreads();
  zadjf_inv2<T, N1, N2, 1>(c, tid, st, 0);
  __syncthreads();
  zadjf_inv1<T, N1, N2, 1>(c, tid, S::NTHR, 1);
  __syncthreads();
  zadjf_inv2<T, N1, N2, 1>(c, tid, st, 1);
  red[tid] = st.bad ? T(-1) : st.umax;
  __syncthreads();
  if (tid < 32) zfast_reduce(c, red, S::NTHR, tid);
  zadjf_fwd1<T, N1, N2, 1>(c, tid, st);
  __syncthreads();
  zadjf_fwd2<T, N1, N2, 1>(c, tid, S::NTHR);
  __syncthreads();
  zadjf_extract<T, N1, N2, 1>(c, tid, S::NTHR);
}

template <typename T, int N1, int N2>
cudaError_t zadv_launch(const ZArgs<T>& a, int nm, cudaStream_t s) {
  using S = ZAdjShape<N1, N2, 1>;
  dim3 grid((S::P + S::Y - 1) / S::Y, S::P, nm);
  const size_t smem = (size_t)S::SM_ELEMS * sizeof(cplx<T>) + (size_t)S::NTHR * sizeof(double);
  k_zadv<T, N1, N2><<<grid, S::NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
cudaError_t zadv_init() {
  return cudaFuncSetAttribute((const void*)k_zadv<T, N1, N2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

template <typename T, int N1, int N2>
size_t zadjf_smem() {
  return (size_t)ZAdjShape<N1, N2>::SM_ELEMS * sizeof(cplx<T>);
}

template <typename T, int N1, int N2>
cudaError_t zadjf_launch(const ZArgs<T>& a, int nm, cudaStream_t s) {
  using S = ZAdjShape<N1, N2>;
  dim3 grid((S::P + S::Y - 1) / S::Y, S::P, nm);
  k_zadjf<T, N1, N2><<<grid, S::NTHR, zadjf_smem<T, N1, N2>(), s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N1, int N2>
cudaError_t zadjf_init() {
  return cudaFuncSetAttribute((const void*)k_zadjf<T, N1, N2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace ns3d

#define NS3D_ZFAST_VARIANT(T, N1, N2)                                                        \
  namespace ns3d {                                                                           \
  template cudaError_t zfast_launch<T, N1, N2>(const ZArgs<T>&, int, cudaStream_t);          \
  template cudaError_t zfast_init<T, N1, N2>();                                              \
  template cudaError_t zrot_launch<T, N1, N2>(const ZArgs<T>&, int, cudaStream_t);           \
  template cudaError_t zrot_init<T, N1, N2>();                                               \
  template cudaError_t zadjf_launch<T, N1, N2>(const ZArgs<T>&, int, cudaStream_t);          \
  template cudaError_t zadjf_init<T, N1, N2>();                                              \
  template cudaError_t zadv_launch<T, N1, N2>(const ZArgs<T>&, int, cudaStream_t);           \
  template cudaError_t zadv_init<T, N1, N2>();                                               \
  }
