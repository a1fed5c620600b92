// CPU emulation of the solver's kernels, block by block with one thread per
// block, for the index-logic tests (tests/test_hostcheck.py).  It runs the
// exact block bodies of ns3d_blocks.cuh with the launch shapes and strides of
// ns3d_geom.h, so a wrong stride, tile bound, padding map or pairing shows up
// against the oracle on the CPU before any GPU run.  Not part of the solver's
// API: the library itself never runs on the host.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ns3d_geom.h"

namespace {

struct HostSync {
  void operator()() const {}
};

template <typename T>
void d1_to_compact(const cplx<T>* d1, cplx<T>* u, int N) {
  const int h = N / 2;
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y)
        for (int z = 0; z < h; ++z) {
          cplx<T> v = d1[(((long long)c * N + x) * N + y) * (h + 1) + z];
          if (x == h || y == h) v = czero<T>();
          u[(((long long)c * N + x) * N + y) * h + z] = v;
        }
}

template <typename T>
void compact_to_d1(const cplx<T>* u, cplx<T>* d1, int N) {
  const int h = N / 2;
  for (int c = 0; c < 3; ++c)
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y)
        for (int z = 0; z <= h; ++z)
          d1[(((long long)c * N + x) * N + y) * (h + 1) + z] =
              z < h ? u[(((long long)c * N + x) * N + y) * h + z] : czero<T>();
}

template <typename T, int SIGN, bool CF1, bool CFL>
void run_col(const ColArgs<T>& a, const ns3d::Launch& L, std::vector<cplx<T>>& sm) {
  for (int z = 0; z < L.gz; ++z)
    for (int y = 0; y < L.gy; ++y)
      for (int x = 0; x < L.gx; ++x)
        colfft_block<T, SIGN, CF1, CFL>(a, x, y, z, 0, 1, sm.data(), HostSync{});
}

template <typename T>
void run_z(const ZArgs<T>& a, const ns3d::Launch& L, std::vector<cplx<T>>& sm) {
  double red[1];
  for (int z = 0; z < L.gz; ++z)
    for (int y = 0; y < L.gy; ++y)
      for (int x = 0; x < L.gx; ++x) zfused_block<T>(a, x, y, z, 0, 1, sm.data(), red, HostSync{});
}

// One evaluation of Algorithm 2 and the spectral step on member 0.
template <typename T>
void rhs_stage(const ns3d::Geom& g, const SpecParams& sp, const cplx<T>* in, cplx<T>* u0,
               cplx<T>* us, cplx<T>* out, int stage, std::vector<cplx<T>>& W1,
               std::vector<cplx<T>>& W2, const std::vector<cplx<T>>& tw, Ns3dCtrl* ctrl,
               std::vector<cplx<T>>& sm) {
  using namespace ns3d;
  run_col<T, +1, true, true>(args_inv_x<T>(g, in, W1.data(), tw.data()), launch_inv_x(g, 1), sm);
  run_col<T, +1, true, false>(args_inv_y<T>(g, W1.data(), W2.data(), tw.data()), launch_inv_y(g, 1), sm);
  run_z<T>(args_z<T>(g, W2.data(), W1.data(), tw.data(), stage == 1 ? ctrl : nullptr), launch_z(g, 1), sm);
  run_col<T, -1, false, true>(args_fwd_y<T>(g, W1.data(), W2.data(), tw.data()), launch_fwd_y(g, 1), sm);
  run_col<T, -1, true, true>(args_fwd_x<T>(g, W2.data(), W1.data(), tw.data()), launch_fwd_x(g, 1), sm);
  SpecArgs<T> s{};
  s.bh = W1.data();
  s.u0 = (stage == 0) ? in : u0;
  s.us = us;
  s.out = out;
  s.N = g.N;
  s.h = g.h;
  s.nmem = 1;
  s.stage = stage;
  s.m6 = g.nBh;
  s.m3 = g.nU;
  s.sp = sp;
  s.ctrl = ctrl;
  const long long total = (long long)g.N * g.N * g.h;
  for (long long i = 0; i < total; ++i) spectral_point<T>(s, i);
}

template <typename T>
int run(int N, int P, const double* prm, const void* uin, void* uout, int nsteps, double dt,
        double* t_out) {
  ns3d::Geom g;
  if (!ns3d::make_geom(N, P, (int)sizeof(cplx<T>), &g)) return 1;
  // prm: L nu s theta eps0 mN_coef q_form cfl
  SpecParams sp = ns3d::make_spec_params(N, P, prm[0], prm[1], prm[2], prm[3], prm[4], prm[5],
                                         (int)prm[6], prm[7], dt);
  std::vector<cplx<T>> tw = ns3d::make_twiddles<T>(P);
  std::vector<cplx<T>> U0(g.nU), US(g.nU), W1(g.nW1), W2(g.nW2);
  size_t sm_elems = std::max(g.smem_c, g.smem_z) / sizeof(cplx<T>) + 16;
  std::vector<cplx<T>> sm(sm_elems);
  d1_to_compact((const cplx<T>*)uin, U0.data(), N);
  Ns3dCtrl ctrl{};
  if (nsteps == 0) {
    rhs_stage<T>(g, sp, U0.data(), nullptr, nullptr, US.data(), 0, W1, W2, tw, &ctrl, sm);
    compact_to_d1(US.data(), (cplx<T>*)uout, N);
    return 0;
  }
  for (int n = 0; n < nsteps; ++n) {
    rhs_stage<T>(g, sp, U0.data(), U0.data(), US.data(), US.data(), 1, W1, W2, tw, &ctrl, sm);
    rhs_stage<T>(g, sp, US.data(), U0.data(), US.data(), US.data(), 2, W1, W2, tw, &ctrl, sm);
    rhs_stage<T>(g, sp, US.data(), U0.data(), US.data(), U0.data(), 3, W1, W2, tw, &ctrl, sm);
  }
  compact_to_d1(U0.data(), (cplx<T>*)uout, N);
  if (t_out) *t_out = ctrl.t;
  return ctrl.status;
}

}  // namespace

extern "C" {

// dtype 0: complex64, 1: complex128.  nsteps = 0: uout = R(uin); nsteps > 0:
// uout = state after nsteps RK3 steps of fixed dt (dt <= 0: CFL).
int ns3d_hostcheck_run(int dtype, int N, int P, const double* prm, const void* uin, void* uout,
                       int nsteps, double dt, double* t_out) {
  if (dtype == 0) return run<float>(N, P, prm, uin, uout, nsteps, dt, t_out);
  return run<double>(N, P, prm, uin, uout, nsteps, dt, t_out);
}

// Radix plan chosen for length n (for tests).
int ns3d_hostcheck_plan(int n, int* radix, int maxp) {
  FftPlanDev pl;
  if (!ns3d::make_fft_plan(n, &pl)) return -1;
  for (int i = 0; i < pl.npass && i < maxp; ++i) radix[i] = pl.radix[i];
  return pl.npass;
}
}
