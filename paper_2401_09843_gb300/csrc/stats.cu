// Ensemble statistics of one level (writers of section 2.4; the empirical
// measure of Algorithm 1 step 3), accumulated in FP64 on the device.
//
// Per member: the energy and enstrophy spectra, the three axis spectra and the
// dissipation rate are histogrammed from the stored coefficients in FP64 with
// compensated (TwoSum/Neumaier) sums merged in a fixed order, so that the
// result is reproducible bit for bit and its error stays a few ulps;
// the second-order structure function follows from the axis spectra,
//   S2(r_j) = (1/3) sum_d sum_k e_d(k) 2 (1 - cos(2 pi k j / N)).
// For the pointwise fields the member's velocity is taken to the N^3 grid
// (unpadded inverse transforms: x, y column passes and a c2r z pass) and a
// Welford update adds it to the pointwise mean and co-moments.
#include <algorithm>
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

// A compensated pair: the value s + c, c holding the rounding errors of the
// additions that made s.
struct CSum {
  double s, c;
};

// Knuth's TwoSum: s = fl(a.s + b.s) and its exact error e = (a.s + b.s) - s,
// folded into the compensation (Neumaier's compensated summation, written for
// pairs so that partial sums merge in any tree).  Commutative, so every lane of
// a butterfly ends with the same pair.
NS3D_HD CSum csum_merge(CSum a, CSum b) {
  const double s = a.s + b.s;
  const double bp = s - a.s;
  const double e = (a.s - (s - bp)) + (b.s - bp);
  return {s, (a.c + b.c) + e};
}

__device__ CSum csum_shfl_down(CSum a, int d) {
  return {__shfl_down_sync(0xffffffffu, a.s, d), __shfl_down_sync(0xffffffffu, a.c, d)};
}

// lane 0 receives the merge of the warp's 32 pairs (a fixed tree)
__device__ CSum csum_warp(CSum a) {
  for (int d = 16; d > 0; d >>= 1) a = csum_merge(a, csum_shfl_down(a, d));
  return a;
}

// one bin of a histogram of pairs: sums in hs, compensations in hc
__device__ void csum_bin_add(double* hs, double* hc, int i, CSum v) {
  const CSum r = csum_merge(CSum{hs[i], hc[i]}, v);
  hs[i] = r.s;
  hc[i] = r.c;
}

// Spectra of one member, one block per kx plane, with compensated sums in a
// fixed order (the result does not depend on scheduling).  Each warp owns a
// histogram of pairs in shared memory and walks rows ky = warp, warp + nw, ...
// 32 kz at a time.  Along a row |k| never decreases with kz, so the lanes
// with one shell K form one run: a segmented suffix merge leaves the run's
// total in its first lane, which alone adds it to the warp's bin K.  The e_z
// bins take one lane each; e_y[ky], e_x[kx] and D are warp merges of lane
// partials.  The warps' histograms are merged in warp order into one pair per
// bin for this plane: part[kx][bin].
template <typename T>
__global__ void k_spectra(const cplx<T>* u, int N, double kscale2, SpecT<double> sp, double2* part) {
  extern __shared__ double sh[];   // [warp][sums HL | compensations HL]
  const int h = N / 2;
  const int L = hist_len(N);
  const int nw = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int i = threadIdx.x; i < 2 * L * nw; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  double* hs = sh + (size_t)warp * 2 * L;
  double* hc = hs + L;
  const int kx = blockIdx.x;
  const int sx = kx < h ? kx : kx - N;
  const long long plane = (long long)N * N * h;
  CSum ex{0.0, 0.0}, dd{0.0, 0.0};   // e_x[kx] (lane 0) and D (per lane)
  for (int ky = warp; ky < N; ky += nw) {
    const int sy = ky < h ? ky : ky - N;
    CSum ey{0.0, 0.0};
    for (int k0 = 0; k0 < h; k0 += 32) {
      const int kz = k0 + lane;
      double e = 0.0, z = 0.0;
      int K = -1;                      // lanes past the row: a run of their own, not stored
      if (kz < h) {
        const long long off = ((long long)kx * N + ky) * h + kz;
        for (int c = 0; c < 3; ++c) {
          const cplx<T> v = u[c * plane + off];
          e += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        if (kz > 0) e *= 2.0;          // the mirror mode -k
        const int k2 = sx * sx + sy * sy + kz * kz;
        K = shell_of(k2);
        z = 0.5 * kscale2 * (double)k2 * e;
        ey = csum_merge(ey, CSum{e, 0.0});
        dd = csum_merge(dd, CSum{lambda_k<double>(k2, sp) * e, 0.0});
        csum_bin_add(hs, hc, 3 * N + kz, CSum{e, 0.0});
      }
      CSum E{0.5 * e, 0.0}, Z{z, 0.0};
      for (int d = 1; d < 32; d <<= 1) {
        const int Ko = __shfl_down_sync(0xffffffffu, K, d);
        const CSum Eo = csum_shfl_down(E, d), Zo = csum_shfl_down(Z, d);
        if (lane + d < 32 && Ko == K) {
          E = csum_merge(E, Eo);
          Z = csum_merge(Z, Zo);
        }
      }
      const int Kp = __shfl_up_sync(0xffffffffu, K, 1);
      if (K >= 0 && (lane == 0 || Kp != K)) {
        csum_bin_add(hs, hc, K, E);
        csum_bin_add(hs, hc, 4 * N + K, Z);
      }
      __syncwarp();
    }
    ey = csum_warp(ey);
    if (lane == 0) {
      csum_bin_add(hs, hc, 2 * N + ky, ey);
      ex = csum_merge(ex, ey);
    }
  }
  dd = csum_warp(dd);
  if (lane == 0) {
    csum_bin_add(hs, hc, N + kx, ex);
    csum_bin_add(hs, hc, 5 * N, dd);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    CSum a{0.0, 0.0};
    for (int w = 0; w < nw; ++w) a = csum_merge(a, CSum{sh[(size_t)w * 2 * L + i], sh[(size_t)w * 2 * L + L + i]});
    part[(size_t)kx * L + i] = make_double2(a.s, a.c);
  }
}

// hist[i] = the planes' pairs part[kx][i] (row length L) merged in kx order,
// rounded once, for i < nout
__global__ void k_spectra_merge(const double2* part, int N, int L, int nout, double* hist) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nout; i += gridDim.x * blockDim.x) {
    CSum a{0.0, 0.0};
    for (int kx = 0; kx < N; ++kx) {
      const double2 q = part[(size_t)kx * L + i];
      a = csum_merge(a, CSum{q.x, q.y});
    }
    hist[i] = a.s + a.c;
  }
}

// ---- ball-averaged structure function
// S2_ball(r_j) = sum_k e_k 2 (1 - jb(q)), jb(q) = 3 (sin q - q cos q) / q^3,
// q = |kappa| r_j = 2 pi j |k| / N (independent of L), e_k = |u_hat_k|^2 summed
// over components and over the mirror mode.  The factor depends on |k|^2 only:
// a table per radius, kBallJ radii per pass over the coefficients.

constexpr int kBallJ = 16;

// Taylor coefficients of 1 - jb(q) in t = q^2:
//   1 - jb = t sum_{n=2}^{15} (-1)^n 6n / (2n+1)! t^(n-2)
// (from sin q - q cos q = sum_{n>=1} (-1)^(n+1) 2n q^(2n+1) / (2n+1)!)
struct BallCoef {
  double c[14];
};

BallCoef ball_coefficients() {
  BallCoef b{};
  double f = 6.0;                                    // (2n+1)! at n = 1
  for (int n = 2; n <= 15; ++n) {
    f *= (double)(2 * n) * (double)(2 * n + 1);
    b.c[n - 2] = ((n % 2) ? -6.0 : 6.0) * n / f;
  }
  return b;
}

// 1 - jb(q): the series (Horner in q^2) below q = 1, where the closed form
// cancels; the closed form above
__device__ double one_minus_jb(double q, const BallCoef& b) {
  if (q < 1.0) {
    const double t = q * q;
    double acc = b.c[13];
#pragma unroll
    for (int n = 12; n >= 0; --n) acc = acc * t + b.c[n];
    return t * acc;
  }
  return 1.0 - 3.0 * (sin(q) - q * cos(q)) / (q * q * q);
}

// G[jj][k2] = 2 (1 - jb(2 pi (j0 + jj) sqrt(k2) / N)), jj < nj, k2 < nk2
__global__ void k_ball_table(double* G, int nk2, int j0, int nj, int N, BallCoef b) {
  const double PI = 3.14159265358979323846;
  const long long total = (long long)nj * nk2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(i / nk2), k2 = (int)(i % nk2);
    const double q = 2.0 * PI * (double)(j0 + jj) * sqrt((double)k2) / (double)N;
    G[i] = 2.0 * one_minus_jb(q, b);
  }
}

// One member, one block per kx plane, 256 threads: per radius jj < nj the
// compensated sum over the plane's modes of e_k G[jj][|k|^2], merged over the
// threads in a fixed order into part[kx][jj].
template <typename T>
__global__ void __launch_bounds__(256) k_s2_ball(const cplx<T>* u, int N, const double* G, int nk2,
                                                 int nj, double2* part) {
  __shared__ double2 sh[8][kBallJ];
  const int h = N / 2;
  const int kx = blockIdx.x;
  const int sx = kx < h ? kx : kx - N;
  const long long plane = (long long)N * N * h;
  CSum acc[kBallJ];
#pragma unroll
  for (int jj = 0; jj < kBallJ; ++jj) acc[jj] = CSum{0.0, 0.0};
  for (int i = threadIdx.x; i < N * h; i += blockDim.x) {
    const int ky = i / h, kz = i % h;
    const long long off = (long long)kx * N * h + i;
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const cplx<T> v = u[c * plane + off];
      e += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    if (kz > 0) e *= 2.0;
    const int sy = ky < h ? ky : ky - N;
    const int k2 = sx * sx + sy * sy + kz * kz;
#pragma unroll
    for (int jj = 0; jj < kBallJ; ++jj)
      if (jj < nj) acc[jj] = csum_merge(acc[jj], CSum{e * G[(size_t)jj * nk2 + k2], 0.0});
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int jj = 0; jj < kBallJ; ++jj) {
    const CSum w = csum_warp(acc[jj]);
    if (lane == 0) sh[warp][jj] = make_double2(w.s, w.c);
  }
  __syncthreads();
  if (threadIdx.x < nj) {
    CSum a{0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x / 32); ++w)
      a = csum_merge(a, CSum{sh[w][threadIdx.x].x, sh[w][threadIdx.x].y});
    part[(size_t)kx * kBallJ + threadIdx.x] = make_double2(a.s, a.c);
  }
}

// warps per k_spectra block: as many histograms of pairs as fit, up to 8
int spectra_warps(int N) {
  const size_t per = 2 * sizeof(double) * (size_t)hist_len(N);
  const size_t nw = (200 * 1024) / per;
  return nw >= 8 ? 8 : (int)nw;
}

// host-side Neumaier sum
struct HostCSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

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
  const int nws = spectra_warps(N);
  if (nws < 1) return NS3D_ERR_NOT_SUPPORTED;
  double* hist = static_cast<double*>(alloc(sizeof(double) * HL * M));
  double2* part = static_cast<double2*>(alloc(sizeof(double2) * HL * (size_t)N));
  const bool ball = out->s2_ball || out->s2_ball_se;
  const int nk2 = 2 * h * h + (h - 1) * (h - 1) + 1;   // |k|^2 <= h^2 + h^2 + (h - 1)^2
  double* G = nullptr;
  double2* partb = nullptr;
  double* s2b = nullptr;
  if (ball) {
    G = static_cast<double*>(alloc(sizeof(double) * kBallJ * (size_t)nk2));
    partb = static_cast<double2*>(alloc(sizeof(double2) * kBallJ * (size_t)N));
    s2b = static_cast<double*>(alloc(sizeof(double) * (size_t)M * (N / 2)));
    if (!G || !partb || !s2b) {
      cleanup();
      return NS3D_ERR_OUT_OF_MEMORY;
    }
  }
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
  if (!hist || !part) {
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
    const size_t sms = 2 * sizeof(double) * (size_t)HL * nws;
    cudaFuncSetAttribute((const void*)k_spectra<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_spectra<T><<<N, 32 * nws, sms, s>>>(u, N, L.sp.kscale * L.sp.kscale, spec_t<double>(L.sp), part);
    k_spectra_merge<<<cdiv(HL, 256), 256, 0, s>>>(part, N, HL, HL, hist + (size_t)m * HL);
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
  std::vector<double> hb;
  if (ball && ok) {
    const BallCoef bc = ball_coefficients();
    for (int j0 = 1; j0 <= N / 2 && ok; j0 += kBallJ) {
      const int nj = std::min(kBallJ, N / 2 - j0 + 1);
      k_ball_table<<<grid_of((long long)nj * nk2), 256, 0, s>>>(G, nk2, j0, nj, N, bc);
      for (int m = 0; m < M; ++m) {
        k_s2_ball<T><<<N, 256, 0, s>>>(U0 + m * g.nU, N, G, nk2, nj, partb);
        k_spectra_merge<<<1, 32, 0, s>>>(partb, N, kBallJ, nj, s2b + (size_t)m * (N / 2) + j0 - 1);
      }
      ok = cudaGetLastError() == cudaSuccess;
    }
    hb.resize((size_t)M * (N / 2));
    ok = ok && cudaMemcpyAsync(hb.data(), s2b, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s) == cudaSuccess;
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
    HostCSum e, z;
    for (int K = 0; K < N; ++K) {
      spec[(size_t)m * N + K] = H[K];
      e.add(H[K]);
      zspec[(size_t)m * N + K] = H[4 * N + K];
      z.add(H[4 * N + K]);
    }
    en[m] = e.value();
    zn[m] = z.value();
    dn[m] = H[5 * N];
    for (int j = 1; j <= N / 2; ++j) {
      HostCSum acc;
      for (int d = 0; d < 3; ++d)
        for (int i = 0; i < N; ++i) {
          const double v = H[(d + 1) * N + i];
          if (v == 0.0) continue;
          const int k = (d < 2 && i >= N / 2) ? i - N : i;
          acc.add(v * 2.0 * (1.0 - std::cos(2.0 * PI * (double)k * j / N)));
        }
      s2[(size_t)m * (N / 2) + j - 1] = acc.value() / 3.0;
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
  if (ball) mean_se(hb, N / 2, out->s2_ball, out->s2_ball_se);
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

// ---------------------------------------------------------------- mesh refinement
// Section 6.1 compares ensembles of one initial measure at two resolutions
// pointwise on the coarse grid x_j = j L / Nc (the fine grid's points with
// index r j, r = Nf / Nc): the error of each sample, of the mean and of the
// variance, and the 1-point Wasserstein distance of the one-point marginals,
// W1(a, b) = integral |F_a(t) - F_b(t)| dt between the empirical CDFs of the
// Ma coarse and Mb fine values at the point, all averaged over the points.

constexpr int kRefineMaxM = 128;    // members per level (values kept per thread)
constexpr int kRefineThreads = 128;
constexpr int kRefineStats = 5;     // W1, |mean diff|, |var diff|, sample error, MC error bar

// fine samples on the coarse points: out[c][j] = in[c][r j] for the three components
template <typename T>
__global__ void k_subsample(const T* in, T* out, int Nf, int Nc) {
  const int r = Nf / Nc;
  const long long n3 = (long long)Nc * Nc * Nc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n3;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / n3);
    const long long j = i % n3;
    const long long x = j / ((long long)Nc * Nc), y = (j / Nc) % Nc, z = j % Nc;
    out[i] = in[(long long)c * Nf * Nf * Nf + ((x * r) * Nf + y * r) * Nf + z * r];
  }
}

__device__ void refine_sort(double* v, int n) {   // insertion sort (n <= kRefineMaxM)
  for (int i = 1; i < n; ++i) {
    const double x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = x;
  }
}

// samples [M][3][n3] (plan dtype); block (b, c) reduces its points of component
// c into part[(c * gridDim.x + b) * kRefineStats + s] as compensated pairs
template <typename T>
__global__ void __launch_bounds__(kRefineThreads) k_refine(const T* sa, int Ma, const T* sb, int Mb,
                                                           long long n3, double2* part) {
  __shared__ double ss[kRefineStats][kRefineThreads], sc[kRefineStats][kRefineThreads];
  const int c = blockIdx.y;
  CSum acc[kRefineStats];
  for (int q = 0; q < kRefineStats; ++q) acc[q] = CSum{0.0, 0.0};
  double a[kRefineMaxM], b[kRefineMaxM];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n3;
       j += (long long)gridDim.x * blockDim.x) {
    double ma = 0.0, mb = 0.0, se = 0.0;
    for (int m = 0; m < Ma; ++m) {
      a[m] = (double)sa[((long long)m * 3 + c) * n3 + j];
      ma += a[m];
    }
    for (int m = 0; m < Mb; ++m) {
      b[m] = (double)sb[((long long)m * 3 + c) * n3 + j];
      mb += b[m];
    }
    if (Ma == Mb) {
      for (int m = 0; m < Ma; ++m) se += fabs(a[m] - b[m]);
      se /= Ma;
    }
    ma /= Ma;
    mb /= Mb;
    double va = 0.0, vb = 0.0;     // two-pass variances (divisor M - 1)
    for (int m = 0; m < Ma; ++m) va += (a[m] - ma) * (a[m] - ma);
    for (int m = 0; m < Mb; ++m) vb += (b[m] - mb) * (b[m] - mb);
    va = Ma > 1 ? va / (Ma - 1) : 0.0;
    vb = Mb > 1 ? vb / (Mb - 1) : 0.0;
    refine_sort(a, Ma);
    refine_sort(b, Mb);
    // integral of |F_a - F_b| over the merged sorted values
    double w = 0.0, prev = a[0] < b[0] ? a[0] : b[0];
    int ia = 0, ib = 0;
    while (ia < Ma || ib < Mb) {
      const bool takea = ib >= Mb || (ia < Ma && a[ia] <= b[ib]);
      const double x = takea ? a[ia] : b[ib];
      w += fabs((double)ia / Ma - (double)ib / Mb) * (x - prev);
      prev = x;
      if (takea) ++ia; else ++ib;
    }
    acc[0] = csum_merge(acc[0], CSum{w, 0.0});
    acc[1] = csum_merge(acc[1], CSum{fabs(ma - mb), 0.0});
    acc[2] = csum_merge(acc[2], CSum{fabs(va - vb), 0.0});
    acc[3] = csum_merge(acc[3], CSum{se, 0.0});
    acc[4] = csum_merge(acc[4], CSum{sqrt(va / Ma + vb / Mb), 0.0});
  }
  for (int q = 0; q < kRefineStats; ++q) {
    ss[q][threadIdx.x] = acc[q].s;
    sc[q][threadIdx.x] = acc[q].c;
  }
  __syncthreads();
  for (int d = kRefineThreads / 2; d > 0; d >>= 1) {
    if (threadIdx.x < d)
      for (int q = 0; q < kRefineStats; ++q) {
        const CSum r = csum_merge(CSum{ss[q][threadIdx.x], sc[q][threadIdx.x]},
                                  CSum{ss[q][threadIdx.x + d], sc[q][threadIdx.x + d]});
        ss[q][threadIdx.x] = r.s;
        sc[q][threadIdx.x] = r.c;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < kRefineStats; ++q)
      part[((long long)c * gridDim.x + blockIdx.x) * kRefineStats + q] = make_double2(ss[q][0], sc[q][0]);
}

template <typename T>
ns3d_status physical_impl(ns3d_plan p, const LevelView& L, int idx, void* out, int on_device,
                          int what);

template <typename T>
ns3d_status refine_impl(ns3d_plan p, const LevelView& Lc, const LevelView& Lf, ns3d_refinement* out) {
  const int Nc = Lc.N, Nf = Lf.N, Ma = Lc.B, Mb = Lf.B;
  const long long n3 = (long long)Nc * Nc * Nc, nf3 = (long long)Nf * Nf * Nf;
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
  auto cleanup = [&]() {
    for (void* q : tmp) cudaFree(q);
  };
  T* sa = static_cast<T*>(alloc(sizeof(T) * 3 * n3 * Ma));
  T* sb = static_cast<T*>(alloc(sizeof(T) * 3 * n3 * Mb));
  T* fine = Nf != Nc ? static_cast<T*>(alloc(sizeof(T) * 3 * nf3)) : nullptr;
  const int nb = (int)std::min<long long>((n3 + kRefineThreads - 1) / kRefineThreads, 152 * 4);
  double2* part = static_cast<double2*>(alloc(sizeof(double2) * 3 * nb * kRefineStats));
  if (!sa || !sb || (Nf != Nc && !fine) || !part) {
    cleanup();
    return NS3D_ERR_OUT_OF_MEMORY;
  }
  ns3d_status st = NS3D_OK;
  for (int m = 0; m < Ma && st == NS3D_OK; ++m)
    st = physical_impl<T>(p, Lc, m, sa + 3 * n3 * m, 1, 0);
  for (int m = 0; m < Mb && st == NS3D_OK; ++m) {
    if (Nf == Nc) {
      st = physical_impl<T>(p, Lf, m, sb + 3 * n3 * m, 1, 0);
    } else {
      st = physical_impl<T>(p, Lf, m, fine, 1, 0);
      if (st == NS3D_OK) {
        k_subsample<T><<<grid_of(3 * n3), 256, 0, s>>>(fine, sb + 3 * n3 * m, Nf, Nc);
        if (cudaGetLastError() != cudaSuccess) st = NS3D_ERR_CUDA;
      }
    }
  }
  std::vector<double2> h(3 * (size_t)nb * kRefineStats);
  if (st == NS3D_OK) {
    k_refine<T><<<dim3(nb, 3), kRefineThreads, 0, s>>>(sa, Ma, sb, Mb, n3, part);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h.data(), part, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = NS3D_ERR_CUDA;
  }
  cleanup();
  if (st != NS3D_OK) return st;
  for (int c = 0; c < 3; ++c) {
    double v[kRefineStats];
    for (int q = 0; q < kRefineStats; ++q) {
      CSum a{0.0, 0.0};
      for (int b = 0; b < nb; ++b) {
        const double2 x = h[((size_t)c * nb + b) * kRefineStats + q];
        a = csum_merge(a, CSum{x.x, x.y});
      }
      v[q] = (a.s + a.c) / (double)n3;
    }
    out->w1[c] = v[0];
    out->mean_err[c] = v[1];
    out->var_err[c] = v[2];
    out->sample_err[c] = Ma == Mb ? v[3] : -1.0;
    out->mc_se[c] = v[4];
  }
  out->coarse_members = Ma;
  out->fine_members = Mb;
  return status_of_level(p, Lc) != NS3D_OK ? status_of_level(p, Lc) : status_of_level(p, Lf);
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

extern "C" ns3d_status ns3d_mesh_refinement(ns3d_plan p, int coarse_N, int fine_N,
                                            ns3d_refinement* out) {
  if (!p || !out || coarse_N <= 0 || fine_N < coarse_N || fine_N % coarse_N) return NS3D_ERR_INVALID_ARG;
  LevelView Lc, Lf;
  if (!find_level(p, coarse_N, &Lc) || !find_level(p, fine_N, &Lf)) return NS3D_ERR_INVALID_ARG;
  if (Lc.B > kRefineMaxM || Lf.B > kRefineMaxM) return NS3D_ERR_NOT_SUPPORTED;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32 ? refine_impl<float>(p, Lc, Lf, out)
                                   : refine_impl<double>(p, Lc, Lf, out);
}

extern "C" ns3d_status ns3d_ensemble_stats(ns3d_plan p, int level_N, ns3d_stats* out) {
  if (!p || !out) return NS3D_ERR_INVALID_ARG;
  LevelView L;
  if (!find_level(p, level_N, &L)) return NS3D_ERR_INVALID_ARG;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32 ? stats_impl<float>(p, L, out) : stats_impl<double>(p, L, out);
}
