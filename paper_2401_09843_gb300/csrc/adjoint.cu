// Discrete adjoint of the SSP-RK3 step and the gradient of a band energy
// (not in the paper; the transpose of its right-hand side, section 2.3, and
// of eq. RK3).  With the stages u, u1, u2 of a step and the adjoint lam of
// its result:
//   a2 = 2/3 (lam + dt J(u2)^T lam)
//   a1 = 1/4 (a2 + dt J(u1)^T a2)
//   lam_n = 1/3 lam + 3/4 a2 + a1 + dt J(u)^T a1,
// J(u)^T w = T_N F[sum_l u_l S_jl(Leray w)] - lambda w (ns3d_blocks.cuh).
// One evaluation of J^T: spectral prep (S from w), inverse x and y of 9
// components (u and S), the adjoint z pass (products; register-resident in
// FP32 at the forward register kernel's sizes, ns3d_zadj.cuh), forward y and
// x of 3 components, and the combine.  dt is the plan's fixed step.
#include <vector>

#include "ns3d.h"
#include "ns3d_launch.h"
#include "plan_internal.h"

using namespace ns3d;

namespace {

template <typename T>
__global__ void k_adj_prep(const cplx<T>* w, cplx<T>* S6, int N, T kscale) {
  const int kx = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N * (N / 2); j += gridDim.x * blockDim.x)
    adj_prep_point<T>(w, S6, N, kscale, kx, j);
}

template <typename T>
__global__ void k_adj_combine(AdjCombineArgs<T> a) {
  const int kx = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.N * (a.N / 2); j += gridDim.x * blockDim.x)
    adj_combine_point<T>(a, kx, j);
}

template <typename T>
__global__ void k_band(const cplx<T>* u, cplx<T>* out, int N, double k_lo, double k_hi) {
  const int kx = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N * (N / 2); j += gridDim.x * blockDim.x)
    band_point<T>(u, out, N, k_lo, k_hi, kx, j);
}

// J = 1/2 sum_{k_lo <= |k| < k_hi} |u_hat_k|^2 over the full spectrum of a
// state in the plan's compact layout [3][kx N][ky N][kz h], one block per kx
// plane: each thread sums its points with Neumaier compensation (Knuth's
// TwoSum of the running sum and each term), then the block merges the
// threads' pairs by a fixed tree in shared memory, so the result does not
// depend on scheduling.  part[kx] = (sum, compensation) of the plane.
struct BandSum {
  double s, c;
};

NS3D_HD BandSum band_sum_merge(BandSum a, BandSum b) {
  const double s = a.s + b.s;
  const double bp = s - a.s;
  const double e = (a.s - (s - bp)) + (b.s - bp);
  return {s, (a.c + b.c) + e};
}

constexpr int kBandThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kBandThreads) k_band_energy(const cplx<T>* u, int N, double k_lo,
                                                              double k_hi, double2* part) {
  __shared__ double ss[kBandThreads], sc[kBandThreads];
  const int h = N / 2;
  const int kx = blockIdx.x;
  const int sx = kx < h ? kx : kx - N;
  const long long plane = (long long)N * N * h;
  BandSum acc{0.0, 0.0};
  if (kx != h) {
    for (int j = threadIdx.x; j < N * h; j += kBandThreads) {
      const int kz = j % h, ky = j / h;
      if (ky == h) continue;
      const int sy = ky < h ? ky : ky - N;
      const double km = sqrt((double)(sx * sx + sy * sy + kz * kz));
      if (!(km >= k_lo && km < k_hi)) continue;
      const long long off = (long long)kx * N * h + j;
      double e = 0.0;
      for (int c = 0; c < 3; ++c) {
        const cplx<T> v = u[c * plane + off];
        e += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
      }
      // 1/2 |u_hat_k|^2, twice for kz > 0 (the mirror mode -k)
      acc = band_sum_merge(acc, BandSum{kz > 0 ? e : 0.5 * e, 0.0});
    }
  }
  ss[threadIdx.x] = acc.s;
  sc[threadIdx.x] = acc.c;
  __syncthreads();
  for (int d = kBandThreads / 2; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      const BandSum r = band_sum_merge(BandSum{ss[threadIdx.x], sc[threadIdx.x]},
                                       BandSum{ss[threadIdx.x + d], sc[threadIdx.x + d]});
      ss[threadIdx.x] = r.s;
      sc[threadIdx.x] = r.c;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[kx] = make_double2(ss[0], sc[0]);
}

template <typename T>
__global__ void k_zadj(ZAdjArgs<T> a) {
  extern __shared__ __align__(16) unsigned char ns3d_smem[];
  zadj_block<T>(a, blockIdx.x, blockIdx.y, threadIdx.x, blockDim.x,
                reinterpret_cast<cplx<T>*>(ns3d_smem), DevSyncS{});
}

dim3 plane_grid(int N) { return dim3((N * (N / 2) + 255) / 256, N); }

// Device buffers of one adjoint computation for one member of a level.
template <typename T>
struct AdjWork {
  const Geom* g = nullptr;
  SpecParams sp{};
  const cplx<T>* tw = nullptr;
  double dt = 0.0;
  std::vector<void*> mem;
  cplx<T>* S6 = nullptr;      // S of w
  cplx<T>* A9 = nullptr;      // 9 x P N h  (inverse x; later Cq3, Bh3)
  cplx<T>* B9 = nullptr;      // 9 x P P h  (inverse y; later Dq3)
  cplx<T>* W1 = nullptr;      // forward-RHS workspaces
  cplx<T>* W2 = nullptr;
  cplx<T>* u[3] = {};         // stage states u, u1, u2
  cplx<T>* a2 = nullptr;
  cplx<T>* a1 = nullptr;
  cplx<T>* tmp = nullptr;
  Ns3dCtrl* ctrl = nullptr;

  cplx<T>* alloc(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(cplx<T>)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.push_back(q);
    return static_cast<cplx<T>*>(q);
  }
  ~AdjWork() {
    for (void* q : mem) cudaFree(q);
  }
  bool init(const LevelView& L, double dt_) {
    g = L.g;
    sp = L.sp;
    tw = static_cast<const cplx<T>*>(L.twP);
    dt = dt_;
    const long long nU = g->nU;
    S6 = alloc(2 * nU);
    A9 = alloc((size_t)9 * g->P * g->N * g->h);
    B9 = alloc((size_t)9 * g->P * g->P * g->h);
    W1 = alloc(g->nW1);
    W2 = alloc(g->nW2);
    for (auto& x : u) x = alloc(nU);
    a2 = alloc(nU);
    a1 = alloc(nU);
    tmp = alloc(nU);
    void* c = nullptr;
    if (cudaMalloc(&c, sizeof(Ns3dCtrl)) != cudaSuccess) return false;
    mem.push_back(c);
    ctrl = static_cast<Ns3dCtrl*>(c);
    return S6 && A9 && B9 && W1 && W2 && u[0] && u[1] && u[2] && a2 && a1 && tmp;
  }
  StageBufs bufs(cplx<T>* u0, cplx<T>* us) const {
    StageBufs b;
    b.g = g;
    b.sp = sp;
    b.W1 = W1;
    b.W2 = W2;
    b.tw = tw;
    b.u0 = u0;
    b.us = us;
    b.ctrl = ctrl;
    return b;
  }
};

#define NS3D_TRY(x)                       \
  do {                                    \
    ns3d_status st_ = (x);                \
    if (st_ != NS3D_OK) return st_;       \
  } while (0)
#define NS3D_CUDA(x)                                  \
  do {                                                \
    if ((x) != cudaSuccess) return NS3D_ERR_CUDA;     \
  } while (0)

// one forward SSP-RK3 step in place on `state` (uses w.tmp as stage buffer)
template <typename T>
ns3d_status forward_step(AdjWork<T>& w, cplx<T>* state, cudaStream_t s) {
  const StageBufs b = w.bufs(state, w.tmp);
  NS3D_TRY(enqueue_rhs<T>(b, 1, 1, state, w.tmp, false, s));
  NS3D_TRY(enqueue_rhs<T>(b, 2, 1, w.tmp, w.tmp, false, s));
  NS3D_TRY(enqueue_rhs<T>(b, 3, 1, w.tmp, state, false, s));
  return NS3D_OK;
}

// the stages of one forward step from u0, each kept in its own buffer: u1 and
// u2 (stages 1 and 2) and, unless `next` is null, u_{n+1} (stage 3)
template <typename T>
ns3d_status forward_stages(AdjWork<T>& w, cplx<T>* u0, cplx<T>* u1, cplx<T>* u2, cplx<T>* next,
                           cudaStream_t s) {
  NS3D_TRY(enqueue_rhs<T>(w.bufs(u0, u1), 1, 1, u0, u1, false, s));
  NS3D_TRY(enqueue_rhs<T>(w.bufs(u0, u1), 2, 1, u1, u2, false, s));
  if (next) NS3D_TRY(enqueue_rhs<T>(w.bufs(u0, u2), 3, 1, u2, next, false, s));
  return NS3D_OK;
}

// bh <- T_N F[sum_l u_l S_jl(Leray w)] (unnormalised), left in w.A9
template <typename T>
ns3d_status adjoint_products(AdjWork<T>& W, const cplx<T>* u, const cplx<T>* w, cudaStream_t s) {
  const Geom& g = *W.g;
  const int P = g.P, N = g.N, h = g.h;
  k_adj_prep<T><<<plane_grid(N), 256, 0, s>>>(w, W.S6, N, (T)W.sp.kscale);
  NS3D_CUDA(cudaGetLastError());
  const long long nA1 = (long long)P * N * h;     // one component after inverse x
  ColArgs<T> ax = args_inv_x<T>(g, u, W.A9, W.tw);
  Launch lx = launch_inv_x(g, 1);                 // 3 components
  NS3D_CUDA(launch_col<T>(ax, COL_INV_CC, lx, s));
  ax.in = W.S6;
  ax.out = W.A9 + 3 * nA1;
  lx.gz = 6;
  NS3D_CUDA(launch_col<T>(ax, COL_INV_CC, lx, s));
  ColArgs<T> ay = args_inv_y<T>(g, W.A9, W.B9, W.tw);
  Launch ly = launch_inv_y(g, 1);
  ly.gz = 9;
  NS3D_CUDA(launch_col<T>(ay, COL_INV_CC, ly, s));
  if (sizeof(T) == 4 && 3 * h == P && zfast_available<float>(P)) {
    // register-resident adjoint z pass (ns3d_zadj.cuh)
    ZArgs<float> za{};
    za.in = reinterpret_cast<const cplx<float>*>(W.B9);
    za.out = reinterpret_cast<cplx<float>*>(W.A9);
    za.tw = reinterpret_cast<const cplx<float>*>(W.tw);
    za.P = P;
    za.h = h;
    za.in_cs = za.out_cs = (long long)P * P * h;
    za.xs = (long long)P * h;
    za.ctrl = nullptr;
    cudaError_t e = cudaErrorInvalidValue;
#define NS3D_ZADJ_GO(A, B) \
    if (P == (A) * (B)) e = zadjf_launch<float, A, B>(za, 1, s);
    NS3D_FOR_ZFAST(NS3D_ZADJ_GO)
#undef NS3D_ZADJ_GO
    NS3D_CUDA(e);
  } else {
    ZAdjArgs<T> az{};
    az.in = W.B9;
    az.out = W.A9;
    az.tw = W.tw;
    az.pl = g.plP;
    az.P = P;
    az.h = h;
    int Wz = 8;
    while (Wz > 2 && (size_t)7 * P * (Wz + 1) * sizeof(cplx<T>) > 200 * 1024) Wz /= 2;
    az.W = Wz;
    az.ldw = Wz + 1;
    const size_t smz = (size_t)7 * P * az.ldw * sizeof(cplx<T>);
    NS3D_CUDA(cudaFuncSetAttribute((const void*)k_zadj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    k_zadj<T><<<dim3(cdiv(P, Wz), P), 128, smz, s>>>(az);
    NS3D_CUDA(cudaGetLastError());
  }
  ColArgs<T> fy = args_fwd_y<T>(g, W.A9, W.B9, W.tw);
  Launch lfy = launch_fwd_y(g, 1);
  lfy.gz = 3;
  NS3D_CUDA(launch_col<T>(fy, COL_FWD_CC, lfy, s));
  ColArgs<T> fx = args_fwd_x<T>(g, W.B9, W.A9, W.tw);
  Launch lfx = launch_fwd_x(g, 1);
  lfx.gz = 3;
  NS3D_CUDA(launch_col<T>(fx, COL_FWD_CC, lfx, s));
  return NS3D_OK;
}

template <typename T>
ns3d_status combine(AdjWork<T>& W, const cplx<T>* w, const cplx<T>* X, const cplx<T>* Y,
                    cplx<T>* out, double alpha, double beta, double gamma, double delta,
                    cudaStream_t s) {
  AdjCombineArgs<T> a{};
  a.bh = W.A9;
  a.w = w;
  a.X = X;
  a.Y = Y;
  a.out = out;
  a.N = W.g->N;
  a.sp = spec_t<T>(W.sp);
  a.dt = (T)W.dt;
  a.alpha = (T)alpha;
  a.beta = (T)beta;
  a.gamma = (T)gamma;
  a.delta = (T)delta;
  k_adj_combine<T><<<plane_grid(W.g->N), 256, 0, s>>>(a);
  NS3D_CUDA(cudaGetLastError());
  return NS3D_OK;
}

// lam_out = adjoint of one step, applied to lam3, given the step's forward
// stage states u = u_n, u1, u2
template <typename T>
ns3d_status adjoint_stages(AdjWork<T>& W, const cplx<T>* u, const cplx<T>* u1, const cplx<T>* u2,
                           const cplx<T>* lam3, cplx<T>* lam_out, cudaStream_t s) {
  // a2 = 2/3 lam + 2/3 dt J(u2)^T lam
  NS3D_TRY(adjoint_products<T>(W, u2, lam3, s));
  NS3D_TRY(combine<T>(W, lam3, nullptr, nullptr, W.a2, 2.0 / 3.0, 2.0 / 3.0, 0, 0, s));
  // a1 = 1/4 a2 + 1/4 dt J(u1)^T a2
  NS3D_TRY(adjoint_products<T>(W, u1, W.a2, s));
  NS3D_TRY(combine<T>(W, W.a2, nullptr, nullptr, W.a1, 0.25, 0.25, 0, 0, s));
  // lam_n = a1 + dt J(u)^T a1 + 1/3 lam + 3/4 a2
  NS3D_TRY(adjoint_products<T>(W, u, W.a1, s));
  NS3D_TRY(combine<T>(W, W.a1, lam3, W.a2, lam_out, 1.0, 1.0, 1.0 / 3.0, 0.75, s));
  return NS3D_OK;
}

// lam_out = adjoint of one step at the forward state un, applied to lam3
// (the stages u1, u2 of the step recomputed from un)
template <typename T>
ns3d_status adjoint_step_c(AdjWork<T>& W, const cplx<T>* un, const cplx<T>* lam3, cplx<T>* lam_out,
                           cudaStream_t s) {
  const long long nU = W.g->nU;
  NS3D_CUDA(cudaMemcpyAsync(W.u[0], un, nU * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s));
  NS3D_CUDA(launch_ctrl_reset(W.ctrl, 1, s));
  NS3D_TRY(forward_stages<T>(W, W.u[0], W.u[1], W.u[2], nullptr, s));
  return adjoint_stages<T>(W, W.u[0], W.u[1], W.u[2], lam3, lam_out, s);
}

size_t d1_elems(int N) { return (size_t)3 * N * N * (N / 2 + 1); }

template <typename T>
ns3d_status d1_in(const void* src, int on_device, cplx<T>* dst, int N, cplx<T>* staging, cudaStream_t s) {
  const void* d = src;
  if (!on_device) {
    NS3D_CUDA(cudaMemcpyAsync(staging, src, d1_elems(N) * sizeof(cplx<T>), cudaMemcpyHostToDevice, s));
    d = staging;
  }
  NS3D_CUDA(launch_d1_to_compact<T>(static_cast<const cplx<T>*>(d), dst, N, s));
  return NS3D_OK;
}

template <typename T>
ns3d_status d1_out(const cplx<T>* src, void* dst, int on_device, int N, cplx<T>* staging, cudaStream_t s) {
  void* d = on_device ? dst : staging;
  NS3D_CUDA(launch_compact_to_d1<T>(src, static_cast<cplx<T>*>(d), N, s));
  if (!on_device)
    NS3D_CUDA(cudaMemcpyAsync(dst, staging, d1_elems(N) * sizeof(cplx<T>), cudaMemcpyDeviceToHost, s));
  return NS3D_OK;
}

template <typename T>
ns3d_status adjoint_step_impl(ns3d_plan p, const LevelView& L, const void* lam1, void* lam0,
                              const void* un, int on_device) {
  const double dt = plan_params(p).dt_fixed;
  if (!(dt > 0)) return NS3D_ERR_NOT_SUPPORTED;
  cudaStream_t s = p_stream(p);
  AdjWork<T> W;
  if (!W.init(L, dt)) return NS3D_ERR_OUT_OF_MEMORY;
  cplx<T>* staging = W.alloc(d1_elems(L.N));
  cplx<T>* lin = W.alloc(W.g->nU);
  cplx<T>* uin = W.alloc(W.g->nU);
  cplx<T>* lo = W.alloc(W.g->nU);
  if (!staging || !lin || !uin || !lo) return NS3D_ERR_OUT_OF_MEMORY;
  NS3D_TRY(d1_in<T>(lam1, on_device, lin, L.N, staging, s));
  NS3D_TRY(d1_in<T>(un, on_device, uin, L.N, staging, s));
  NS3D_TRY(adjoint_step_c<T>(W, uin, lin, lo, s));
  NS3D_TRY(d1_out<T>(lo, lam0, on_device, L.N, staging, s));
  NS3D_CUDA(cudaStreamSynchronize(s));
  return NS3D_OK;
}

template <typename T>
ns3d_status grad_impl(ns3d_plan p, const LevelView& L, int idx, double k_lo, double k_hi,
                      int nsteps, int C, void* grad, int on_device) {
  const double dt = plan_params(p).dt_fixed;
  if (!(dt > 0)) return NS3D_ERR_NOT_SUPPORTED;
  // C <= 0: one segment whose stage states all come from the forward pass
  const bool keep_all = C <= 0;
  if (keep_all) C = nsteps > 0 ? nsteps : 1;
  cudaStream_t s = p_stream(p);
  AdjWork<T> W;
  if (!W.init(L, dt)) return NS3D_ERR_OUT_OF_MEMORY;
  const long long nU = W.g->nU;
  const int nck = (nsteps + C - 1) / C;
  // checkpoints (every C-th state), and the stage states u_n, u1, u2 of each
  // step of one segment at seg + 3 i nU
  cplx<T>* ck = keep_all ? nullptr : W.alloc((size_t)(nck > 0 ? nck : 1) * nU);
  cplx<T>* seg = W.alloc((size_t)3 * C * nU);
  cplx<T>* state = W.alloc(nU);
  cplx<T>* lam = W.alloc(nU);
  cplx<T>* lam2 = W.alloc(nU);
  cplx<T>* staging = W.alloc(d1_elems(L.N));
  if ((!keep_all && !ck) || !seg || !state || !lam || !lam2 || !staging)
    return NS3D_ERR_OUT_OF_MEMORY;
  auto stage_buf = [&](int i, int j) { return seg + ((size_t)3 * i + j) * nU; };
  NS3D_CUDA(launch_ctrl_reset(W.ctrl, 1, s));
  NS3D_CUDA(cudaMemcpyAsync(state, static_cast<const cplx<T>*>(L.U0) + (size_t)idx * nU,
                            nU * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s));
  if (keep_all) {
    NS3D_CUDA(cudaMemcpyAsync(stage_buf(0, 0), state, nU * sizeof(cplx<T>),
                              cudaMemcpyDeviceToDevice, s));
    for (int n = 0; n < nsteps; ++n)
      NS3D_TRY(forward_stages<T>(W, stage_buf(n, 0), stage_buf(n, 1), stage_buf(n, 2),
                                 n + 1 < nsteps ? stage_buf(n + 1, 0) : state, s));
  } else {
    for (int n = 0; n < nsteps; ++n) {
      if (n % C == 0)
        NS3D_CUDA(cudaMemcpyAsync(ck + (size_t)(n / C) * nU, state, nU * sizeof(cplx<T>),
                                  cudaMemcpyDeviceToDevice, s));
      NS3D_TRY(forward_step<T>(W, state, s));
    }
  }
  // lam(T) = dJ/du(T) = u(T) on the band
  k_band<T><<<plane_grid(L.N), 256, 0, s>>>(state, lam, L.N, k_lo, k_hi);
  NS3D_CUDA(cudaGetLastError());
  for (int sgi = nck - 1; sgi >= 0; --sgi) {
    const int start = sgi * C, end = (start + C < nsteps) ? start + C : nsteps;
    if (!keep_all) {
      // recompute the segment from its checkpoint, keeping every stage state
      NS3D_CUDA(launch_ctrl_reset(W.ctrl, 1, s));
      NS3D_CUDA(cudaMemcpyAsync(stage_buf(0, 0), ck + (size_t)sgi * nU, nU * sizeof(cplx<T>),
                                cudaMemcpyDeviceToDevice, s));
      for (int i = 0; i < end - start; ++i)
        NS3D_TRY(forward_stages<T>(W, stage_buf(i, 0), stage_buf(i, 1), stage_buf(i, 2),
                                   i + 1 < end - start ? stage_buf(i + 1, 0) : nullptr, s));
    }
    for (int n = end - 1; n >= start; --n) {
      const int i = n - start;
      NS3D_TRY(adjoint_stages<T>(W, stage_buf(i, 0), stage_buf(i, 1), stage_buf(i, 2), lam, lam2, s));
      cplx<T>* t = lam;
      lam = lam2;
      lam2 = t;
    }
  }
  NS3D_TRY(d1_out<T>(lam, grad, on_device, L.N, staging, s));
  NS3D_CUDA(cudaStreamSynchronize(s));
  return NS3D_OK;
}

template <typename T>
ns3d_status band_energy_impl(ns3d_plan p, const LevelView& L, int idx, double k_lo, double k_hi,
                             double* J) {
  cudaStream_t s = p_stream(p);
  const long long nU = L.g->nU;
  double2* part = nullptr;
  NS3D_CUDA(cudaMalloc(&part, (size_t)L.N * sizeof(double2)));
  k_band_energy<T><<<L.N, kBandThreads, 0, s>>>(static_cast<const cplx<T>*>(L.U0) + (size_t)idx * nU,
                                                 L.N, k_lo, k_hi, part);
  cudaError_t e = cudaGetLastError();
  std::vector<double2> h(L.N);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, (size_t)L.N * sizeof(double2),
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return NS3D_ERR_CUDA;
  BandSum tot{0.0, 0.0};
  for (int kx = 0; kx < L.N; ++kx) tot = band_sum_merge(tot, BandSum{h[kx].x, h[kx].y});
  *J = tot.s + tot.c;
  return status_of_level(p, L);
}

}  // namespace

extern "C" ns3d_status ns3d_band_energy(ns3d_plan p, int member, double k_lo, double k_hi,
                                        double* J) {
  LevelView L;
  int idx;
  if (!p || !J || !(k_hi > k_lo) || !member_view(p, member, &L, &idx)) return NS3D_ERR_INVALID_ARG;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32 ? band_energy_impl<float>(p, L, idx, k_lo, k_hi, J)
                                   : band_energy_impl<double>(p, L, idx, k_lo, k_hi, J);
}

extern "C" ns3d_status ns3d_adjoint_step(ns3d_plan p, int member, const void* lambda_np1,
                                         void* lambda_n, const void* uhat_n, int on_device) {
  LevelView L;
  int idx;
  if (!p || !lambda_np1 || !lambda_n || !uhat_n || !member_view(p, member, &L, &idx))
    return NS3D_ERR_INVALID_ARG;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32 ? adjoint_step_impl<float>(p, L, lambda_np1, lambda_n, uhat_n, on_device)
                                   : adjoint_step_impl<double>(p, L, lambda_np1, lambda_n, uhat_n, on_device);
}

extern "C" ns3d_status ns3d_grad_band_energy(ns3d_plan p, int member, double k_lo, double k_hi,
                                             int nsteps, int checkpoint_every, void* grad,
                                             int on_device) {
  LevelView L;
  int idx;
  if (!p || !grad || nsteps < 0 || !(k_hi > k_lo) || !member_view(p, member, &L, &idx))
    return NS3D_ERR_INVALID_ARG;
  PlanDeviceGuard dg(p);
  return plan_dtype(p) == NS3D_F32
             ? grad_impl<float>(p, L, idx, k_lo, k_hi, nsteps, checkpoint_every, grad, on_device)
             : grad_impl<double>(p, L, idx, k_lo, k_hi, nsteps, checkpoint_every, grad, on_device);
}
