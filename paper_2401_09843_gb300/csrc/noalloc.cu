// Allocation-free evaluation of the time derivative for small grids.
//
// Some callers cannot allocate device memory at the moment they need the
// right-hand side: real-time or embedded hosts that fix their device memory
// budget at start-up, plug-in hosts whose allocator must not be re-entered
// from a callback, and latency-bound loops that cannot afford the implicit
// device synchronisation of cudaMalloc/cudaFree.  ns3d_eval_rhs_noalloc
// serves them: it takes the input and
// output buffers from the caller and keeps every intermediate array of the
// evaluation in one file-scope device array (g_noalloc_scratch below), which
// every GPU that loads this library holds until the process exits.  It calls no
// cudaMalloc, cudaFree or other allocating routine.
//
// Limits: N <= 32 (padded size P <= 48) in FP32 or FP64; the arrays of one
// evaluation then need at most 6.4 MiB (N = 32, FP64) of the 8 MiB array.  Every call
// shares the one array and leaves the last call's intermediates in it: calls
// whose work overlaps on the GPU (two streams, or two host threads) race and
// corrupt each other's results; order them on one stream.  Nothing in the
// array has to start at zero: each pass writes every element the next pass
// reads.
#include <mutex>

#include "ns3d.h"
#include "ns3d_launch.h"

using namespace ns3d;

namespace {

constexpr int kNoAllocMaxN = 32;
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, looked up once per device (by the first call
// on that device) and kept for the life of the process: a cudaDeviceReset of
// that device invalidates it, after which this entry point must not be called
// again.  In host code the name g_noalloc_scratch is only a host-side
// stand-in, never a device address.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

ns3d_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return NS3D_ERR_NOT_SUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NS3D_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return NS3D_OK;
}

template <typename T>
__global__ void k_noalloc_twiddles(cplx<T>* tw, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    double s, c;
    sincospi(2.0 * e / n, &s, &c);
    tw[e].x = (T)c;
    tw[e].y = (T)(-s);
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
ns3d_status run(const Geom& g, const SpecParams& sp, const void* uhat, void* rhs, void* base,
                cudaStream_t s) {
  const size_t esz = sizeof(cplx<T>);
  unsigned char* p = static_cast<unsigned char*>(base);
  cplx<T>* U = reinterpret_cast<cplx<T>*>(p);
  p += align256(g.nU * esz);
  cplx<T>* W1 = reinterpret_cast<cplx<T>*>(p);
  p += align256(g.nW1 * esz);
  cplx<T>* W2 = reinterpret_cast<cplx<T>*>(p);
  p += align256(g.nW2 * esz);
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(p);
  if (kernels_init<T>() != cudaSuccess) return NS3D_ERR_CUDA;
  k_noalloc_twiddles<T><<<(g.P + 127) / 128, 128, 0, s>>>(tw, g.P);
  if (cudaGetLastError() != cudaSuccess) return NS3D_ERR_CUDA;
  if (launch_d1_to_compact<T>(static_cast<const cplx<T>*>(uhat), U, g.N, s) != cudaSuccess ||
      launch_col<T>(args_inv_x<T>(g, U, W1, tw), COL_INV_CC, launch_inv_x(g, 1), s) != cudaSuccess ||
      launch_col<T>(args_inv_y<T>(g, W1, W2, tw), COL_INV_CC, launch_inv_y(g, 1), s) != cudaSuccess ||
      launch_zpass<T>(args_z<T>(g, W2, W1, tw, nullptr), g, 1, s) != cudaSuccess ||
      launch_col<T>(args_fwd_y<T>(g, W1, W2, tw), COL_FWD_CC, launch_fwd_y(g, 1), s) != cudaSuccess ||
      launch_col<T>(args_fwd_x<T>(g, W2, W1, tw), COL_FWD_CC, launch_fwd_x(g, 1), s) != cudaSuccess)
    return NS3D_ERR_CUDA;
  SpecArgs<T> a{};
  a.bh = W1;
  a.u0 = U;
  a.us = U;
  a.out = U;
  a.N = g.N;
  a.h = g.h;
  a.nmem = 1;
  a.stage = 0;
  a.m6 = g.nBh;
  a.m3 = g.nU;
  a.sp = spec_t<T>(sp);
  a.ctrl = nullptr;
  if (launch_spectral<T>(a, s) != cudaSuccess ||
      launch_compact_to_d1<T>(U, static_cast<cplx<T>*>(rhs), g.N, s) != cudaSuccess)
    return NS3D_ERR_CUDA;
  return NS3D_OK;
}

}  // namespace

extern "C" ns3d_status ns3d_eval_rhs_noalloc(int N, ns3d_dtype dtype, const ns3d_params* prm,
                                             const void* uhat, void* rhs_out, void* cuda_stream) {
  if (!prm || !uhat || !rhs_out || (dtype != NS3D_F32 && dtype != NS3D_F64))
    return NS3D_ERR_INVALID_ARG;
  if (N < 4 || N % 2 || N > kNoAllocMaxN) return NS3D_ERR_INVALID_ARG;
  const ns3d_params& P = *prm;
  if (!(P.L > 0) || !(P.nu >= 0) || !(P.s >= 0.5) || !(P.theta > 0) || !(P.eps0 >= 0) ||
      !(P.mN_coef >= 0) || (P.q_form != 0 && P.q_form != 1) || P.n_pad < -1)
    return NS3D_ERR_INVALID_ARG;
  if (P.nonlinear_form != 0) return NS3D_ERR_NOT_SUPPORTED;
  // n_pad 0 and -1 both take the smallest 7-smooth size >= 3N/2 (no benchmark here)
  int Pad = P.n_pad > 0 ? P.n_pad : default_padded_size(N);
  if (2 * Pad < 3 * N || Pad > 3 * kNoAllocMaxN / 2) return NS3D_ERR_INVALID_ARG;
  const int esz = dtype == NS3D_F32 ? 8 : 16;
  Geom g;
  if (!make_geom(N, Pad, esz, &g)) return NS3D_ERR_NOT_SUPPORTED;
  const size_t need = align256(g.nU * esz) + align256(g.nW1 * esz) + align256(g.nW2 * esz) +
                      align256((size_t)Pad * esz);
  if (need > kNoAllocScratchBytes) return NS3D_ERR_INVALID_ARG;
  const SpecParams sp = make_spec_params(N, Pad, P.L, P.nu, P.s, P.theta, P.eps0, P.mN_coef,
                                         P.q_form, P.cfl, P.dt_fixed);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return NS3D_ERR_CUDA;
  }
  void* base = nullptr;
  ns3d_status st = scratch_address(dev, &base);
  if (st != NS3D_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return dtype == NS3D_F32 ? run<float>(g, sp, uhat, rhs_out, base, s)
                           : run<double>(g, sp, uhat, rhs_out, base, s);
}
