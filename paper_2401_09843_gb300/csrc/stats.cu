// Ensemble statistics of one level (writers of section 2.4; the empirical
// measure of Algorithm 1 step 3), accumulated in FP64 on the device.
//
// Per member: the energy spectrum and the three axis spectra are histogrammed
// from the stored coefficients (FP64 block histograms, atomics across blocks);
// the second-order structure function follows from the axis spectra,
//   S2(r_j) = (1/3) sum_d sum_k e_d(k) 2 (1 - cos(2 pi k j / N)).
// For the pointwise fields the member's velocity is taken to the N^3 grid
// (unpadded inverse transforms: x, y column passes and a c2r z pass) and a
// Welford update adds it to the pointwise mean and co-moments.
#include <cmath>
#include <vector>

#include "ns3d.h"
#include "ns3d_launch.h"
#include "plan_internal.h"

using namespace ns3d;

namespace {

// per-member histogram rows: [0, N) E(K); [N, 4N) the axis spectra e_x, e_y,
// e_z; [4N, 5N) Z(K); [5N] D = sum lambda_k |u_hat_k|^2 (full spectrum)
NS3D_HDC int hist_len(int N) { return 5 * N + 1; }

template <typename T>
__global__ void k_spectra(const cplx<T>* u, int N, double kscale2, SpecT<double> sp, double* hist) {
  extern __shared__ double sh[];
  const int h = N / 2;
  const int L = hist_len(N);
  for (int i = threadIdx.x; i < L; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const int kx = blockIdx.x;
  for (int j = threadIdx.x; j < N * h; j += blockDim.x) {
    const int ky = j / h, kz = j % h;
    const long long plane = (long long)N * N * h;
    const long long off = ((long long)kx * N + ky) * h + kz;
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const cplx<T> v = u[c * plane + off];
      e += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    if (kz > 0) e *= 2.0;     // the mirror mode -k
    if (e == 0.0) continue;
    const int sx = kx < h ? kx : kx - N;
    const int sy = ky < h ? ky : ky - N;
    const int k2 = sx * sx + sy * sy + kz * kz;
    const int K = shell_of(k2);
    atomicAdd(&sh[K], 0.5 * e);
    atomicAdd(&sh[2 * N + ky], e);
    atomicAdd(&sh[3 * N + kz], e);
    atomicAdd(&sh[N + kx], e);
    atomicAdd(&sh[4 * N + K], 0.5 * kscale2 * (double)k2 * e);
    atomicAdd(&sh[5 * N], lambda_k<double>(k2, sp) * e);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L; i += blockDim.x)
    if (sh[i] != 0.0) atomicAdd(&hist[i], sh[i]);
}

template <typename T>
__global__ void k_zinv(ZInvArgs<T> a) {
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  zinv_block<T>(a, blockIdx.x, blockIdx.y, threadIdx.x, blockDim.x,
                reinterpret_cast<cplx<T>*>(ns3d_smem), DevSyncS{});
}

template <typename T>
__global__ void k_welford(const T* u, long long N3, int n, double* mean, double* C) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x)
    welford_point<T>(u, N3, i, n, mean, C);
}

// second moments E[u_i u_j] = C_ij / M + mean_i mean_j (in place over C) and
// variances C_ii / (M - 1) into var
__global__ void k_finalize(const double* mean, double* C, double* var, long long N3, int M) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x) {
    int q = 0;
    for (int r = 0; r < 3; ++r)
      for (int s = r; s < 3; ++s, ++q) {
        const double c = C[q * N3 + i];
        if (r == s) var[r * N3 + i] = M > 1 ? c / (M - 1) : 0.0;
        C[q * N3 + i] = c / M + mean[r * N3 + i] * mean[s * N3 + i];
      }
  }
}

int grid_of(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g));
}

template <typename T>
ns3d_status stats_impl(ns3d_plan p, LevelView& L, ns3d_stats* out) {
  const Geom& g = *L.g;
  const int N = g.N, h = g.h, M = L.B;
  const long long N3 = (long long)N * N * N;
  cudaStream_t s = p_stream(p);
  const bool fields = out->mean || out->second || out->var;
  if (fields && g.plN.npass == 0) return NS3D_ERR_NOT_SUPPORTED;
  std::vector<void*> tmp;
  auto alloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    tmp.push_back(q);
    return q;
  };
  auto cleanup = [&]() {
    for (void* q : tmp) cudaFree(q);
  };
  const int HL = hist_len(N);
  double* hist = static_cast<double*>(alloc(sizeof(double) * HL * M));
  cplx<T>* twN = nullptr;
  double *mean = nullptr, *C = nullptr, *var = nullptr;
  T* phys = nullptr;
  cplx<T>* A = nullptr;
  cplx<T>* Bq = nullptr;
  if (fields) {
    twN = static_cast<cplx<T>*>(alloc(sizeof(cplx<T>) * N));
    mean = static_cast<double*>(alloc(sizeof(double) * 3 * N3));
    C = static_cast<double*>(alloc(sizeof(double) * 6 * N3));
    var = static_cast<double*>(alloc(sizeof(double) * 3 * N3));
    phys = static_cast<T*>(alloc(sizeof(T) * 3 * N3));
    A = static_cast<cplx<T>*>(alloc(sizeof(cplx<T>) * 3 * (size_t)N * N * h));
    Bq = static_cast<cplx<T>*>(alloc(sizeof(cplx<T>) * 3 * (size_t)N * N * h));
    if (!twN || !mean || !C || !var || !phys || !A || !Bq) {
      cleanup();
      return NS3D_ERR_OUT_OF_MEMORY;
    }
  }
  if (!hist) {
    cleanup();
    return NS3D_ERR_OUT_OF_MEMORY;
  }
  bool ok = cudaMemsetAsync(hist, 0, sizeof(double) * HL * M, s) == cudaSuccess;
  if (fields) {
    std::vector<cplx<T>> tw = make_twiddles<T>(N);
    ok = ok && cudaMemcpyAsync(twN, tw.data(), sizeof(cplx<T>) * N, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(mean, 0, sizeof(double) * 3 * N3, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(C, 0, sizeof(double) * 6 * N3, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;   // tw lives on the host stack
  }
  const cplx<T>* U0 = static_cast<const cplx<T>*>(L.U0);
  for (int m = 0; m < M && ok; ++m) {
    const cplx<T>* u = U0 + m * g.nU;
    k_spectra<T><<<N, 256, sizeof(double) * HL, s>>>(u, N, L.sp.kscale * L.sp.kscale,
                                                      spec_t<double>(L.sp), hist + (size_t)m * HL);
    ok = cudaGetLastError() == cudaSuccess;
    if (!fields || !ok) continue;
    // inverse x and y without padding (n = N): column passes of the generic engine
    ColArgs<T> ax = args_inv_x<T>(g, u, A, twN);
    ax.pl = g.plN; ax.nrow_out = N; ax.W = g.WcN; ax.ldw = g.ldwcN;
    ax.out_bs = (long long)N * N * h;
    Launch lx{cdiv((long long)N * h, g.WcN), 1, 3, g.nthr_c, g.smem_cN};
    ColArgs<T> ay = args_inv_y<T>(g, A, Bq, twN);
    ay.pl = g.plN; ay.nrow_out = N; ay.W = g.WcN; ay.ldw = g.ldwcN;
    ay.in_bs = (long long)N * N * h; ay.out_bs = (long long)N * N * h; ay.out_os = (long long)N * h;
    Launch ly{cdiv(h, g.WcN), N, 3, g.nthr_c, g.smem_cN};
    ok = launch_col<T>(ax, COL_INV_CC, lx, s) == cudaSuccess &&
         launch_col<T>(ay, COL_INV_CC, ly, s) == cudaSuccess;
    if (!ok) break;
    ZInvArgs<T> az{};
    az.in = Bq; az.out = phys; az.tw = twN; az.pl = g.plN; az.N = N; az.h = h;
    az.W = 8; az.ldw = 9;
    const size_t smz = (size_t)4 * N * az.ldw * sizeof(cplx<T>);
    cudaFuncSetAttribute((const void*)k_zinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_zinv<T><<<dim3(cdiv(N, az.W), N), 128, smz, s>>>(az);
    k_welford<T><<<grid_of(N3), 256, 0, s>>>(phys, N3, m + 1, mean, C);
    ok = cudaGetLastError() == cudaSuccess;
  }
  std::vector<double> hh((size_t)HL * M);
  ok = ok && cudaMemcpyAsync(hh.data(), hist, sizeof(double) * hh.size(), cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (fields && ok) {
    k_finalize<<<grid_of(N3), 256, 0, s>>>(mean, C, var, N3, M);
    ok = cudaGetLastError() == cudaSuccess;
    if (ok && out->mean) ok = cudaMemcpyAsync(out->mean, mean, sizeof(double) * 3 * N3, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok && out->second) ok = cudaMemcpyAsync(out->second, C, sizeof(double) * 6 * N3, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    if (ok && out->var) ok = cudaMemcpyAsync(out->var, var, sizeof(double) * 3 * N3, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  cleanup();
  if (!ok) return NS3D_ERR_CUDA;

  // per-member scalars and spectra -> Monte Carlo means and standard errors
  const double PI = 3.14159265358979323846;
  std::vector<double> spec((size_t)M * N), zspec((size_t)M * N), s2((size_t)M * (N / 2)), en(M),
      zn(M), dn(M);
  for (int m = 0; m < M; ++m) {
    const double* H = &hh[(size_t)m * HL];
    double e = 0.0, z = 0.0;
    for (int K = 0; K < N; ++K) {
      spec[(size_t)m * N + K] = H[K];
      e += H[K];
      zspec[(size_t)m * N + K] = H[4 * N + K];
      z += H[4 * N + K];
    }
    en[m] = e;
    zn[m] = z;
    dn[m] = H[5 * N];
    for (int j = 1; j <= N / 2; ++j) {
      double acc = 0.0;
      for (int d = 0; d < 3; ++d)
        for (int i = 0; i < N; ++i) {
          const double v = H[(d + 1) * N + i];
          if (v == 0.0) continue;
          const int k = (d < 2 && i >= N / 2) ? i - N : i;
          acc += v * 2.0 * (1.0 - std::cos(2.0 * PI * (double)k * j / N));
        }
      s2[(size_t)m * (N / 2) + j - 1] = acc / 3.0;
    }
  }
  auto mean_se = [&](const std::vector<double>& x, int n, double* mu, double* se) {
    for (int k = 0; k < n; ++k) {
      double mm = 0.0, q = 0.0;
      for (int m = 0; m < M; ++m) {     // Welford over members
        const double v = x[(size_t)m * n + k], d = v - mm;
        mm += d / (m + 1);
        q += d * (v - mm);
      }
      if (mu) mu[k] = mm;
      if (se) se[k] = M > 1 ? std::sqrt(q / (M - 1) / M) : 0.0;
    }
  };
  mean_se(spec, N, out->spectrum, out->spectrum_se);
  mean_se(s2, N / 2, out->s2, out->s2_se);
  mean_se(zspec, N, out->enstrophy_spectrum, out->enstrophy_spectrum_se);
  double emu = 0.0, ese = 0.0;
  mean_se(en, 1, &emu, &ese);
  out->energy = emu;
  out->energy_se = ese;
  mean_se(zn, 1, &out->enstrophy, &out->enstrophy_se);
  mean_se(dn, 1, &out->dissipation, &out->dissipation_se);
  out->members = M;
  return status_of_level(p, L);
}

// omega_hat = i kappa x u_hat on the compact layout
template <typename T>
__global__ void k_curl(const cplx<T>* u, cplx<T>* w, int N, T kscale) {
  const int h = N / 2;
  const long long plane = (long long)N * N * h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(i % h);
    const int ky = (int)((i / h) % N), kx = (int)(i / ((long long)h * N));
    const T ax = kscale * T(kx < h ? kx : kx - N), ay = kscale * T(ky < h ? ky : ky - N),
            az = kscale * T(kz);
    const cplx<T> u0 = u[i], u1 = u[plane + i], u2 = u[2 * plane + i];
    // (kappa x u)_c, then times i: i (a + ib) = -b + ia
    const cplx<T> c0 = ay * u2 - az * u1, c1 = az * u0 - ax * u2, c2 = ax * u1 - ay * u0;
    w[i] = cmake(-c0.y, c0.x);
    w[plane + i] = cmake(-c1.y, c1.x);
    w[2 * plane + i] = cmake(-c2.y, c2.x);
  }
}

template <typename T>
__global__ void k_magnitude(const T* v, T* out, long long N3) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N3;
       i += (long long)gridDim.x * blockDim.x) {
    const T a = v[i], b = v[N3 + i], c = v[2 * N3 + i];
    out[i] = sqrt(a * a + b * b + c * c);
  }
}

// what = 0: the velocity [3][N][N][N]; what = 1: |omega| [N][N][N]
template <typename T>
ns3d_status physical_impl(ns3d_plan p, const LevelView& L, int idx, void* out, int on_device,
                          int what) {
  const Geom& g = *L.g;
  const int N = g.N, h = g.h;
  const long long N3 = (long long)N * N * N;
  if (g.plN.npass == 0) return NS3D_ERR_NOT_SUPPORTED;
  cudaStream_t s = p_stream(p);
  std::vector<void*> tmp;
  auto alloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    tmp.push_back(q);
    return q;
  };
  const size_t nc = 3 * (size_t)N * N * h;
  cplx<T>* twN = static_cast<cplx<T>*>(alloc(sizeof(cplx<T>) * N));
  cplx<T>* W = static_cast<cplx<T>*>(alloc(sizeof(cplx<T>) * nc));
  cplx<T>* A = static_cast<cplx<T>*>(alloc(sizeof(cplx<T>) * nc));
  // phys: the three components on the grid; mag: the result ([3][N^3] velocity
  // written in place, or [N^3] |omega|); the caller's device buffer when it has one
  const long long nout = what == 0 ? 3 * N3 : N3;
  T* mag = on_device ? static_cast<T*>(out) : static_cast<T*>(alloc(sizeof(T) * nout));
  T* phys = what == 0 ? mag : static_cast<T*>(alloc(sizeof(T) * 3 * N3));
  bool ok = twN && W && A && phys && mag;
  if (ok) {
    std::vector<cplx<T>> tw = make_twiddles<T>(N);
    const cplx<T>* u = static_cast<const cplx<T>*>(L.U0) + idx * g.nU;
    ok = cudaMemcpyAsync(twN, tw.data(), sizeof(cplx<T>) * N, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
    if (what == 1) k_curl<T><<<grid_of((long long)N * N * h), 256, 0, s>>>(u, W, N, T(L.sp.kscale));
    else ok = ok && cudaMemcpyAsync(W, u, sizeof(cplx<T>) * nc, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
    // inverse x and y without padding, then c2r along z: as for the statistics
    ColArgs<T> ax = args_inv_x<T>(g, W, A, twN);
    ax.pl = g.plN; ax.nrow_out = N; ax.W = g.WcN; ax.ldw = g.ldwcN;
    ax.out_bs = (long long)N * N * h;
    Launch lx{cdiv((long long)N * h, g.WcN), 1, 3, g.nthr_c, g.smem_cN};
    ColArgs<T> ay = args_inv_y<T>(g, A, W, twN);
    ay.pl = g.plN; ay.nrow_out = N; ay.W = g.WcN; ay.ldw = g.ldwcN;
    ay.in_bs = (long long)N * N * h; ay.out_bs = (long long)N * N * h; ay.out_os = (long long)N * h;
    Launch ly{cdiv(h, g.WcN), N, 3, g.nthr_c, g.smem_cN};
    ok = ok && cudaGetLastError() == cudaSuccess && launch_col<T>(ax, COL_INV_CC, lx, s) == cudaSuccess &&
         launch_col<T>(ay, COL_INV_CC, ly, s) == cudaSuccess;
    if (ok) {
      ZInvArgs<T> az{};
      az.in = W; az.out = phys; az.tw = twN; az.pl = g.plN; az.N = N; az.h = h;
      az.W = 8; az.ldw = 9;
      const size_t smz = (size_t)4 * N * az.ldw * sizeof(cplx<T>);
      cudaFuncSetAttribute((const void*)k_zinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      k_zinv<T><<<dim3(cdiv(N, az.W), N), 128, smz, s>>>(az);
      if (what == 1) k_magnitude<T><<<grid_of(N3), 256, 0, s>>>(phys, mag, N3);
      ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok && !on_device)
      ok = cudaMemcpyAsync(out, mag, sizeof(T) * nout, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  }
  for (void* q : tmp) cudaFree(q);
  if (!(twN && W && A && phys && mag)) return NS3D_ERR_OUT_OF_MEMORY;
  return ok ? NS3D_OK : NS3D_ERR_CUDA;
}

ns3d_status physical_entry(ns3d_plan p, int member, void* out, int on_device, int what) {
  if (!p || !out) return NS3D_ERR_INVALID_ARG;
  LevelView L;
  int idx = 0;
  if (!member_view(p, member, &L, &idx)) return NS3D_ERR_INVALID_ARG;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32 ? physical_impl<float>(p, L, idx, out, on_device, what)
                                   : physical_impl<double>(p, L, idx, out, on_device, what);
}

}  // namespace

extern "C" ns3d_status ns3d_vorticity_magnitude(ns3d_plan p, int member, void* out, int on_device) {
  return physical_entry(p, member, out, on_device, 1);
}

extern "C" ns3d_status ns3d_physical_field(ns3d_plan p, int member, void* out, int on_device) {
  return physical_entry(p, member, out, on_device, 0);
}

extern "C" ns3d_status ns3d_ensemble_stats(ns3d_plan p, int level_N, ns3d_stats* out) {
  if (!p || !out) return NS3D_ERR_INVALID_ARG;
  LevelView L;
  if (!find_level(p, level_N, &L)) return NS3D_ERR_INVALID_ARG;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32 ? stats_impl<float>(p, L, out) : stats_impl<double>(p, L, out);
}
