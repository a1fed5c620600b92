// Host-side planning shared by the CUDA plan (plan.cu) and the CPU block
// emulator (hostcheck.cpp): radix plans, twiddle tables, array sizes, tile
// widths and launch shapes of every pass of one ensemble level.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <vector>

#include "ns3d_blocks.cuh"

namespace ns3d {

// Largest-first radix choice over the radices the generic engine dispatches on.
inline bool make_fft_plan(int n, FftPlanDev* pl) {
  static const int radices[] = {16, 12, 8, 7, 6, 5, 4, 3, 2};
  pl->n = n;
  pl->npass = 0;
  if (n < 2) return false;
  int m = n;
  while (m > 1) {
    int pick = 0;
    for (int r : radices)
      if (m % r == 0) { pick = r; break; }
    if (!pick || pl->npass == NS3D_MAX_PASSES) return false;
    pl->radix[pl->npass++] = pick;
    m /= pick;
  }
  return true;
}

inline bool is_7_smooth(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

inline int default_padded_size(int N) {
  int P = (3 * N + 1) / 2;
  while (!is_7_smooth(P)) ++P;
  return P;
}

// tw[e] = exp(-2 pi i e / n), computed in long double.
template <typename T>
std::vector<cplx<T>> make_twiddles(int n) {
  std::vector<cplx<T>> t(n);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int e = 0; e < n; ++e) {
    const long double a = 2.0L * pi * (long double)e / (long double)n;
    t[e].x = (T)std::cos(a);
    t[e].y = (T)(-std::sin(a));
  }
  return t;
}

// Geometry of one level: sizes in complex elements per member, tiles, launches.
struct Geom {
  int N = 0, h = 0, P = 0;
  int esz = 0;                 // bytes of one complex element
  long long nU = 0, nA = 0, nBq = 0, nCq = 0, nDq = 0, nBh = 0, nW1 = 0, nW2 = 0;
  FftPlanDev plP{}, plN{};
  int Wc = 0, ldwc = 0, nthr_c = 256;   // column passes of length P
  size_t smem_c = 0;
  int WcN = 0, ldwcN = 0;               // column passes of length N (statistics)
  size_t smem_cN = 0;
  int Wz = 0, ldwz = 0, nthr_z = 128;   // fused z pass
  size_t smem_z = 0;
  int form = 0;                          // nonlinear form (0 divergence, 1 advective, 2 rotational)
  int Wzf = 0, ldwzf = 0, nthr_zf = 128; // z pass of forms 1 and 2
  size_t smem_zf = 0;
};

constexpr size_t kSmemTarget = 113 * 1024;   // two blocks per SM
constexpr size_t kSmemMax = 227 * 1024;      // one block per SM

inline int col_width(int n, int npass, int esz, int W0, size_t* smem) {
  int W = W0;
  auto need = [&](int w) { return npass >= 2 ? (size_t)2 * n * (w + 1) * esz : (size_t)0; };
  while (W > 1 && need(W) > kSmemTarget) W /= 2;
  *smem = need(W);
  return W;
}

inline bool make_geom(int N, int P, int esz, Geom* g) {
  if (N < 4 || N % 2 || P < N) return false;
  g->N = N;
  g->h = N / 2;
  g->P = P;
  g->esz = esz;
  const long long n = N, p = P, h = N / 2;
  g->nU = 3 * n * n * h;
  g->nA = 3 * p * n * h;
  g->nBq = 3 * p * h * p;
  g->nCq = 6 * p * h * p;
  g->nDq = 6 * p * n * h;
  g->nBh = 6 * n * n * h;
  g->nW1 = std::max(g->nA, std::max(g->nCq, g->nBh));
  g->nW2 = std::max(g->nBq, g->nDq);
  if (!make_fft_plan(P, &g->plP)) return false;
  // length-N transforms serve only the statistics; npass = 0 marks them unavailable
  if (!make_fft_plan(N, &g->plN)) g->plN.npass = 0;
  const int W0 = esz == 8 ? 16 : 8;
  g->Wc = col_width(P, g->plP.npass, esz, W0, &g->smem_c);
  // long FP32 lines: fewer than 4 columns (16-byte row segments) at two blocks
  // per SM; take 4 columns at one block of 512 threads instead
  if (esz == 8 && g->Wc < 4 && g->plP.npass >= 2 && (size_t)2 * P * 5 * esz <= kSmemMax) {
    g->Wc = 4;
    g->smem_c = (size_t)2 * P * 5 * esz;
    g->nthr_c = 512;
  }
  g->ldwc = g->Wc + 1;
  g->WcN = g->plN.npass ? col_width(N, g->plN.npass, esz, W0, &g->smem_cN) : 1;
  g->ldwcN = g->WcN + 1;
  int Wz = esz == 8 ? 8 : 4;
  auto needz = [&](int w) { return (size_t)4 * P * (w + 1) * esz + (size_t)8 * g->nthr_z; };
  while (Wz > 2 && needz(Wz) > kSmemTarget) Wz /= 2;
  // one block per SM anyway: FP32 runs 512 threads instead of 128
  if (esz == 8 && needz(Wz) > kSmemTarget) g->nthr_z = 512;
  g->Wz = Wz;
  g->ldwz = Wz + 1;
  g->smem_z = needz(Wz);
  return true;
}

// Forms 1 and 2 of the nonlinear term: workspaces for the form's nf fields
// (W1: nf P^2 h after the inverse y pass; W2: nf P N h after the inverse x
// pass, 3 P^2 h after the z pass) and the zform_block tile (W y columns,
// zform_buffers(form) shared lines of P (W + 1) elements).
inline bool set_form_geom(Geom* g, int form) {
  g->form = form;
  if (form == 0) return true;
  const long long n = g->N, p = g->P, h = g->h;
  const long long nf = form_fields(form);
  g->nW1 = std::max(g->nW1, nf * p * p * h);
  g->nW2 = std::max(g->nW2, std::max(nf * p * n * h, 3 * p * p * h));
  const int nb = zform_buffers(form);
  auto need = [&](int w, int nthr) {
    return (size_t)nb * g->P * (w + 1) * g->esz + (size_t)8 * nthr;
  };
  int W = g->esz == 8 ? 4 : 8;
  while (W > 1 && need(W, 128) > kSmemTarget) W /= 2;
  // one block per SM anyway: FP32 runs 512 threads instead of 128
  const int nthr = (g->esz == 8 && need(W, 128) > kSmemTarget) ? 512 : 128;
  if (need(W, nthr) > kSmemMax) return false;
  g->Wzf = W;
  g->ldwzf = W + 1;
  g->nthr_zf = nthr;
  g->smem_zf = need(W, nthr);
  return true;
}

// Tile shapes the zform kernel can run at for this level: W y columns per
// block (1 .. 16) and 128, 256 or 512 threads (FP32; FP64 kernels are built
// for 128), within the shared memory of one block.  Every shape computes the
// same values (each column's transforms do not depend on the tile); plan
// creation times them and keeps the fastest.
struct FormTile {
  int W, nthr;
  size_t smem;
};

inline std::vector<FormTile> form_tile_candidates(const Geom& g) {
  std::vector<FormTile> c;
  if (g.form == 0) return c;
  const int nb = zform_buffers(g.form);
  for (int W = 1; W <= 16; W *= 2)
    for (int nthr = 128; nthr <= (g.esz == 8 ? 512 : 128); nthr *= 2) {
      const size_t need = (size_t)nb * g.P * (W + 1) * g.esz + (size_t)8 * nthr;
      if (need <= kSmemMax && W <= g.P) c.push_back({W, nthr, need});
    }
  return c;
}

inline void set_form_tile(Geom* g, const FormTile& t) {
  g->Wzf = t.W;
  g->ldwzf = t.W + 1;
  g->nthr_zf = t.nthr;
  g->smem_zf = t.smem;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- pass arguments

// Inverse x: U [m][3][N][N*h] -> A [m][3][P][N*h]
template <typename T>
ColArgs<T> args_inv_x(const Geom& g, const cplx<T>* in, cplx<T>* out, const cplx<T>* tw) {
  ColArgs<T> a{};
  a.in = in; a.out = out; a.tw = tw; a.pl = g.plP;
  a.h = g.h; a.nrow_in = g.N; a.nrow_out = g.P; a.pad_in = 1; a.trunc_out = 0;
  a.ncols = g.N * g.h; a.W = g.Wc; a.ldw = g.ldwc;
  a.in_bs = (long long)g.N * g.N * g.h; a.in_os = 0; a.in_cs = 1; a.in_rs = (long long)g.N * g.h;
  a.out_bs = (long long)g.P * g.N * g.h; a.out_os = 0; a.out_cs = 1; a.out_rs = (long long)g.N * g.h;
  a.scale = T(1);
  return a;
}

// Inverse y: A [m][3][P][N][h] -> Bq [m][3][P][P][h]
template <typename T>
ColArgs<T> args_inv_y(const Geom& g, const cplx<T>* in, cplx<T>* out, const cplx<T>* tw) {
  ColArgs<T> a{};
  a.in = in; a.out = out; a.tw = tw; a.pl = g.plP;
  a.h = g.h; a.nrow_in = g.N; a.nrow_out = g.P; a.pad_in = 1; a.trunc_out = 0;
  a.ncols = g.h; a.W = g.Wc; a.ldw = g.ldwc;
  a.in_bs = (long long)g.P * g.N * g.h; a.in_os = (long long)g.N * g.h; a.in_cs = 1; a.in_rs = g.h;
  a.out_bs = (long long)g.P * g.P * g.h; a.out_os = (long long)g.P * g.h; a.out_cs = 1; a.out_rs = g.h;
  a.scale = T(1);
  return a;
}

// Forward y: Cq [m][6][P][P][h] -> Dq [m][6][P][N][h]
template <typename T>
ColArgs<T> args_fwd_y(const Geom& g, const cplx<T>* in, cplx<T>* out, const cplx<T>* tw) {
  ColArgs<T> a{};
  a.in = in; a.out = out; a.tw = tw; a.pl = g.plP;
  a.h = g.h; a.nrow_in = g.P; a.nrow_out = g.N; a.pad_in = 0; a.trunc_out = 1;
  a.ncols = g.h; a.W = g.Wc; a.ldw = g.ldwc;
  a.in_bs = (long long)g.P * g.P * g.h; a.in_os = (long long)g.P * g.h; a.in_cs = 1; a.in_rs = g.h;
  a.out_bs = (long long)g.P * g.N * g.h; a.out_os = (long long)g.N * g.h; a.out_cs = 1; a.out_rs = g.h;
  a.scale = T(1);
  return a;
}

// Forward x: Dq [m][6][P][N*h] -> Bh [m][6][N][N*h]
template <typename T>
ColArgs<T> args_fwd_x(const Geom& g, const cplx<T>* in, cplx<T>* out, const cplx<T>* tw) {
  ColArgs<T> a{};
  a.in = in; a.out = out; a.tw = tw; a.pl = g.plP;
  a.h = g.h; a.nrow_in = g.P; a.nrow_out = g.N; a.pad_in = 0; a.trunc_out = 1;
  a.ncols = g.N * g.h; a.W = g.Wc; a.ldw = g.ldwc;
  a.in_bs = (long long)g.P * g.N * g.h; a.in_os = 0; a.in_cs = 1; a.in_rs = (long long)g.N * g.h;
  a.out_bs = (long long)g.N * g.N * g.h; a.out_os = 0; a.out_cs = 1; a.out_rs = (long long)g.N * g.h;
  a.scale = T(1);
  return a;
}

template <typename T>
ZArgs<T> args_z(const Geom& g, const cplx<T>* in, cplx<T>* out, const cplx<T>* tw, Ns3dCtrl* ctrl) {
  ZArgs<T> a{};
  a.in = in; a.out = out; a.tw = tw; a.pl = g.plP;
  a.P = g.P; a.h = g.h; a.W = g.Wz; a.ldw = g.ldwz;
  a.in_bs = g.nBq; a.in_cs = (long long)g.P * g.P * g.h;
  a.out_bs = g.nCq; a.out_cs = (long long)g.P * g.P * g.h;
  a.xs = (long long)g.P * g.h;
  a.ctrl = ctrl;
  return a;
}

struct Launch {
  int gx, gy, gz, nthr;
  size_t smem;
};

inline Launch launch_inv_x(const Geom& g, int nm) { return {cdiv((long long)g.N * g.h, g.Wc), 1, nm * 3, g.nthr_c, g.smem_c}; }
inline Launch launch_inv_y(const Geom& g, int nm) { return {cdiv(g.h, g.Wc), g.P, nm * 3, g.nthr_c, g.smem_c}; }
inline Launch launch_z(const Geom& g, int nm) { return {cdiv(g.P, g.Wz), g.P, nm, g.nthr_z, g.smem_z}; }
inline Launch launch_fwd_y(const Geom& g, int nm) { return {cdiv(g.h, g.Wc), g.P, nm * 6, g.nthr_c, g.smem_c}; }
inline Launch launch_fwd_x(const Geom& g, int nm) { return {cdiv((long long)g.N * g.h, g.Wc), 1, nm * 6, g.nthr_c, g.smem_c}; }

// Spectral parameters of the level (eq. shv_disc constants, CFL)
inline SpecParams make_spec_params(int N, int P, double L, double nu, double s, double theta,
                                   double eps0, double mN_coef, int q_form, double cfl,
                                   double dt_fixed) {
  SpecParams sp{};
  const double pi = 3.14159265358979323846;
  sp.kscale = 2.0 * pi / L;
  sp.nu = nu;
  sp.s = s;
  sp.epsN = eps0 * std::pow((double)N, 1.0 - 2.0 * s);
  sp.mN2 = mN_coef * mN_coef * std::pow((double)N, 2.0 * theta);
  sp.qexp = (2.0 * s - 1.0) / (2.0 * theta);
  sp.kthr = (int)std::floor(sp.mN2 * (1.0 + 1e-12));
  sp.q_form = q_form;
  sp.inv_P3 = 1.0 / ((double)P * P * P);
  sp.cfl = cfl;
  sp.dx = L / N;
  sp.dt_fixed = dt_fixed;
  // largest damping rate over the retained set (|k_i| <= N/2 - 1)
  const int hm = N / 2 - 1;
  double lmax = 0.0;
  for (int k2 = 0; k2 <= 3 * hm * hm; ++k2) {
    const double kap2 = sp.kscale * sp.kscale * k2;
    double lam = nu * kap2;
    if (k2 > sp.kthr && k2 > 0) {
      double q = q_form == 0 ? 1.0 - std::pow(sp.mN2 / k2, sp.qexp) : 1.0;
      lam += sp.epsN * std::pow(kap2, s) * q;
    }
    if (lam > lmax) lmax = lam;
  }
  sp.lam_max = lmax;
  return sp;
}

}  // namespace ns3d
