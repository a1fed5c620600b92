// CPU emulation of the solver's kernels, block by block with one thread per
// block, for the index-logic tests (tests/test_abi_host.py).  It runs the
// exact block bodies of ns3d_blocks.cuh with the launch shapes and strides of
// ns3d_geom.h, so a wrong stride, tile bound, padding map or pairing shows up
// against the oracle on the CPU before any GPU run.  Not part of the solver's
// API: the library itself never runs on the host.
#include <algorithm>
#include <cstring>
#include <limits>
#include <vector>

#include "ns3d_geom.h"
#include "ns3d_zfast.cuh"
#include "ns3d_colfast.cuh"
#include "ns3d_xfused.cuh"
#include "ns3d_colfast3.cuh"
#include "ns3d_zfast3.cuh"
#include "ns3d_zrot.cuh"
#include "ns3d_zadj.cuh"

namespace {

// 0: generic kernels only; 1: the register-resident kernels the GPU uses;
// 2: as 1 but the three-pass kernels at the test factorisations below
int g_use_fast = 1;

// nonlinear form of the emulated right-hand side (0 divergence, 1 advective,
// 2 rotational)
int g_form = 0;
// > 0: the zform tile width W instead of the default shape (any shape the
// plan's tuner may pick must compute the same values)
int g_form_W = 0;

// three-pass factorisations emulated at short lengths (the GPU builds them
// for long lines only), so that their index logic meets the oracle
#define NS3D_FOR_LONG_TEST(X) X(4, 3, 4) X(6, 4, 4) X(8, 4, 6) X(8, 6, 8)

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

template <typename T, int SIGN, int N1, int N2>
void run_colfast(const ColArgs<T>& a, const ns3d::Launch& L) {
  using S = ColFastShape<N1, N2>;
  std::vector<cplx<T>> sm(S::SM_ELEMS);
  const int gx = (a.ncols + S::W - 1) / S::W;
  for (int z = 0; z < L.gz; ++z)
    for (int y = 0; y < L.gy; ++y)
      for (int x = 0; x < gx; ++x) {
        colfast_twiddles<T, SIGN, N1, N2>(sm.data(), a.tw, 0, 1);
        for (int t = 0; t < S::NTHR; ++t)
          colfast_pass1<T, SIGN, N1, N2, (SIGN > 0)>(a, x, y, z, t, S::NTHR, sm.data(), sm.data() + S::P);
        for (int t = 0; t < S::NTHR; ++t)
          colfast_pass2<T, SIGN, N1, N2, (SIGN < 0)>(a, x, y, z, t, S::NTHR, sm.data() + S::P);
      }
}

template <typename T, int SIGN, int N1, int N2, int N3>
void run_colfast3(const ColArgs<T>& a, int gy, int gz) {
  using S = ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>;
  std::vector<cplx<LongC<T>>> sm(S::SM_ELEMS);
  const int gx = (a.ncols + S::W - 1) / S::W;
  for (int z = 0; z < gz; ++z)
    for (int y = 0; y < gy; ++y)
      for (int x = 0; x < gx; ++x) {
        const int ncol = std::min(S::W, a.ncols - x * S::W);
        for (int t = 0; t < S::NTHR; ++t) colfast3_twiddles<T, SIGN, S::P>(sm.data(), a.tw, t, S::NTHR);
        cplx<LongC<T>>* X = sm.data() + S::P;
        for (int t = 0; t < S::NTHR; ++t)
          colfast3_pass1<T, SIGN, N1, N2, N3, (SIGN > 0)>(a, x, y, z, t, S::NTHR, sm.data(), X);
        for (int t = 0; t < S::NTHR; ++t) colfast3_pass2<T, SIGN, N1, N2, N3>(t, S::NTHR, ncol, sm.data(), X);
        for (int t = 0; t < S::NTHR; ++t)
          colfast3_pass3<T, SIGN, N1, N2, N3, (SIGN < 0)>(a, x, y, z, t, S::NTHR, X);
      }
}

template <typename T, int SIGN, bool CF1, bool CFL>
void run_col(const ColArgs<T>& a, const ns3d::Launch& L, std::vector<cplx<T>>& sm) {
  const bool padded_inverse = SIGN > 0 && a.pad_in && !a.trunc_out && a.nrow_in == 2 * a.h;
  const bool truncated_forward = SIGN < 0 && !a.pad_in && a.trunc_out && a.nrow_out == 2 * a.h;
  if (g_use_fast && 3 * a.h == a.pl.n && (padded_inverse || truncated_forward)) {
#define NS3D_HC_CF3(A, B, C)                              \
    if (a.pl.n == (A) * (B) * (C)) {                      \
      run_colfast3<T, SIGN, A, B, C>(a, L.gy, L.gz);      \
      return;                                             \
    }
    if (sizeof(T) == 4) {
      NS3D_FOR_COLFAST3(NS3D_HC_CF3)
    } else {        // FP64: the three-pass kernels in double-single arithmetic
      NS3D_FOR_COLFAST3_F64(NS3D_HC_CF3)
    }
    if (g_use_fast == 2) {
      NS3D_FOR_LONG_TEST(NS3D_HC_CF3)
    }
#undef NS3D_HC_CF3
  }
  if (g_use_fast && sizeof(T) == 4 && a.W == 16 && 3 * a.h == a.pl.n &&
      (padded_inverse || truncated_forward)) {
#define NS3D_HC_CF(A, B)                        \
    if (a.pl.n == (A) * (B)) {                  \
      run_colfast<T, SIGN, A, B>(a, L);         \
      return;                                   \
    }
    NS3D_FOR_COLFAST(NS3D_HC_CF)
#undef NS3D_HC_CF
  }
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

// The adjoint right-hand side's register-resident z pass, phase by phase and
// thread by thread, on x rows by < nx.
template <typename T, int N1, int N2>
void run_zadjf(const ZArgs<T>& a, int nx) {
  using S = ZAdjShape<N1, N2>;
  std::vector<cplx<T>> sm(S::SM_ELEMS);
  std::vector<ZAdjState<T, N1, N2>> st(S::NTHR);
  const int gx = (S::P + S::Y - 1) / S::Y;
  for (int by = 0; by < nx; ++by)
    for (int bx = 0; bx < gx; ++bx) {
      ZFastCtx<T, N1, N2> c = zadjf_ctx<T, N1, N2>(a, bx, by, 0, sm.data());
      for (int t = 0; t < S::NTHR; ++t) zfast_load_twiddles(c, t, S::NTHR);
      for (int part = 0; part < 2; ++part) {
        for (int t = 0; t < S::NTHR; ++t) zadjf_inv1(c, t, S::NTHR, part);
        for (int t = 0; t < S::NTHR; ++t) zadjf_inv2(c, t, st[t], part);
      }
      for (int t = 0; t < S::NTHR; ++t) zadjf_fwd1(c, t, st[t]);
      for (int t = 0; t < S::NTHR; ++t) zadjf_fwd2(c, t, S::NTHR);
      for (int t = 0; t < S::NTHR; ++t) zadjf_extract(c, t, S::NTHR);
    }
}

// The rotational form's register-resident z pass, phase by phase and thread
// by thread.
template <typename T, int N1, int N2>
void run_zrot(const ZArgs<T>& a, int nm) {
  using S = ZRotShape<N1, N2>;
  std::vector<cplx<T>> sm(S::SM_ELEMS);
  std::vector<T> red(S::NTHR);
  std::vector<ZFastState<T, N1, N2>> st(S::NTHR);
  const int gx = (S::P + S::Y - 1) / S::Y;
  for (int bz = 0; bz < nm; ++bz)
    for (int by = 0; by < S::P; ++by)
      for (int bx = 0; bx < gx; ++bx) {
        ZFastCtx<T, N1, N2> c = zrot_ctx<T, N1, N2>(a, bx, by, bz, sm.data());
        for (int t = 0; t < S::NTHR; ++t) zfast_load_twiddles(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) zrot_inv1(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) {
          zrot_inv2(c, t, st[t]);
          red[t] = st[t].bad ? T(-1) : st[t].umax;
        }
        zfast_reduce(c, red.data(), S::NTHR, 0);
        for (int t = 0; t < S::NTHR; ++t) zrot_fwd1(c, t, st[t]);
        for (int t = 0; t < S::NTHR; ++t) zrot_fwd2(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) zrot_extract(c, t, S::NTHR);
      }
}

// The advective form's register-resident z pass, phase by phase and thread
// by thread.
template <typename T, int N1, int N2>
void run_zadv(const ZArgs<T>& a, int nm) {
  using S = ZAdjShape<N1, N2, 1>;
  std::vector<cplx<T>> sm(S::SM_ELEMS);
  std::vector<T> red(S::NTHR);
  std::vector<ZAdjState<T, N1, N2>> st(S::NTHR);
  const int gx = (S::P + S::Y - 1) / S::Y;
  for (int bz = 0; bz < nm; ++bz)
    for (int by = 0; by < S::P; ++by)
      for (int bx = 0; bx < gx; ++bx) {
        ZFastCtx<T, N1, N2> c = zadjf_ctx<T, N1, N2, 1>(a, bx, by, bz, sm.data());
        for (int t = 0; t < S::NTHR; ++t) zfast_load_twiddles(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) zadjf_inv1<T, N1, N2, 1>(c, t, S::NTHR, 0);
        for (int t = 0; t < S::NTHR; ++t) zadjf_inv2<T, N1, N2, 1>(c, t, st[t], 0);
        for (int t = 0; t < S::NTHR; ++t) zadjf_inv1<T, N1, N2, 1>(c, t, S::NTHR, 1);
        for (int t = 0; t < S::NTHR; ++t) {
          zadjf_inv2<T, N1, N2, 1>(c, t, st[t], 1);
          red[t] = st[t].bad ? T(-1) : st[t].umax;
        }
        zfast_reduce(c, red.data(), S::NTHR, 0);
        for (int t = 0; t < S::NTHR; ++t) zadjf_fwd1<T, N1, N2, 1>(c, t, st[t]);
        for (int t = 0; t < S::NTHR; ++t) zadjf_fwd2<T, N1, N2, 1>(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) zadjf_extract<T, N1, N2, 1>(c, t, S::NTHR);
      }
}

template <typename T>
void run_zform(const ZArgs<T>& a, int form, const ns3d::Launch& L, std::vector<cplx<T>>& sm) {
  double red[1];
  for (int z = 0; z < L.gz; ++z)
    for (int y = 0; y < L.gy; ++y)
      for (int x = 0; x < L.gx; ++x)
        zform_block<T>(a, form, x, y, z, 0, 1, sm.data(), red, HostSync{});
}

// The register-resident z pass, phase by phase and thread by thread.
template <typename T, int N1, int N2>
void run_zfast(const ZArgs<T>& a, int nm) {
  using S = ZFastShape<N1, N2>;
  std::vector<cplx<T>> sm(S::SM_ELEMS);
  std::vector<T> red(S::NTHR);
  std::vector<ZFastState<T, N1, N2>> st(S::NTHR);
  const int gx = (S::P + S::Y - 1) / S::Y;
  for (int bz = 0; bz < nm; ++bz)
    for (int by = 0; by < S::P; ++by)
      for (int bx = 0; bx < gx; ++bx) {
        ZFastCtx<T, N1, N2> c = zfast_ctx<T, N1, N2>(a, bx, by, bz, sm.data());
        for (int t = 0; t < S::NTHR; ++t) zfast_load_twiddles(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) zfast_inv1(c, t, S::NTHR);
        for (int t = 0; t < S::NTHR; ++t) {
          zfast_inv2(c, t, st[t]);
          red[t] = st[t].bad ? T(-1) : st[t].umax;
        }
        zfast_reduce(c, red.data(), S::NTHR, 0);
        for (int r = 0; r < 2; ++r) {
          for (int t = 0; t < S::NTHR; ++t) zfast_fwd1(c, t, st[t], r);
          for (int t = 0; t < S::NTHR; ++t) zfast_fwd2(c, t, S::NTHR);
          for (int t = 0; t < S::NTHR; ++t) zfast_extract(c, t, r);
        }
      }
}

// The three-pass z pass as one persistent block running every tile (rows
// x < nx of each member), phase by phase and thread by thread.
template <typename T, int N1, int N2, int N3>
void run_zfast3(const ZArgs<T>& a, int nm, int nx) {
  using S = ZFast3Shape<N1, N2, N3>;
  using C = LongC<T>;
  std::vector<cplx<C>> sm(S::SM_ELEMS);
  std::vector<T> red(S::NTHR);
  std::vector<ZFast3State<T, N1, N2, N3>> st(S::NTHR);
  for (int t = 0; t < S::NTHR; ++t) zfast3_twiddles<T, N1, N2, N3>(a, sm.data(), t, S::NTHR);
  for (auto& x : st) {
    x.umax = C(0);
    x.chk = C(0);
  }
  int cur = -1;
  auto flush = [&]() {
    if (cur < 0 || !a.ctrl) return;
    for (int t = 0; t < S::NTHR; ++t) red[t] = zfast3_red_value(st[t]);
    zfast3_flush<T>(a, cur, red.data(), S::NTHR, 0);
  };
  const long long ntiles = (long long)nm * S::P * (S::P / 2);
  for (long long t = 0; t < ntiles; ++t) {
    int bz, by, y0;
    zfast3_tile<N1, N2, N3>(t, &bz, &by, &y0);
    if (by >= nx) continue;
    if (bz != cur) {
      flush();
      for (auto& x : st) {
        x.umax = T(0);
        x.chk = T(0);
      }
      cur = bz;
    }
    const ZFast3Ctx<T, N1, N2, N3> c = zfast3_ctx<T, N1, N2, N3>(a, bz, by, y0, sm.data());
    for (int i = 0; i < S::NTHR; ++i) zfast3_inv1(c, i, S::NTHR);
    for (int i = 0; i < S::NTHR; ++i) zfast3_inv2(c, i, S::NTHR);
    for (int i = 0; i < S::NTHR; ++i) zfast3_inv3(c, i, st[i]);
    for (int r = 0; r < 2; ++r) {
      for (int i = 0; i < S::NTHR; ++i) zfast3_fwdA(c, i, st[i], r);
      for (int i = 0; i < S::NTHR; ++i) zfast3_fwdB(c, i, S::NTHR);
      for (int i = 0; i < S::NTHR; ++i) zfast3_fwdC(c, i, S::NTHR);
      for (int i = 0; i < S::NTHR; ++i) zfast3_extract(c, i, S::NTHR, r);
    }
  }
  flush();
}

template <typename T>
bool run_z_fast_if_any(const ZArgs<T>& a, int P) {
  if (3 * a.h != P) return false;
#define NS3D_HC_ZF3(A, B, C)           \
  if (P == (A) * (B) * (C)) {          \
    run_zfast3<T, A, B, C>(a, 1, P);   \
    return true;                       \
  }
  if (sizeof(T) == 4) {
    NS3D_FOR_ZFAST3(NS3D_HC_ZF3)
  } else {          // FP64: the three-pass kernels in double-single arithmetic
    NS3D_FOR_ZFAST3_F64(NS3D_HC_ZF3)
  }
  if (g_use_fast == 2) {
    NS3D_FOR_LONG_TEST(NS3D_HC_ZF3)
  }
  if (sizeof(T) != 4) return false;
#undef NS3D_HC_ZF3
#define NS3D_HC_ZF(A, B)               \
  if (P == (A) * (B)) {                \
    run_zfast<T, A, B>(a, 1);          \
    return true;                       \
  }
  NS3D_FOR_ZFAST(NS3D_HC_ZF)
#undef NS3D_HC_ZF
  return false;
}

// The fused x pass, phase by phase and thread by thread, on member 0.  The
// staging ring is filled at the same points as the kernel's tile loads (a
// copy lands at once), after the slots were poisoned with NaN, so a phase
// that read a slot before its tile or after its reuse shows in the result.
template <typename T, int N1, int N2>
void run_xfused(const XFusedArgs<T>& a) {
  using S = XFusedShape<N1, N2>;
  std::vector<cplx<T>> sm(S::SM_ELEMS);
  cplx<T>* ring = sm.data();
  cplx<T>* tw = ring + S::OFF_TW;
  cplx<T>* X = ring + S::OFF_X;
  std::vector<XFusedState<T, N1, N2>> st(S::NTHR);
  std::vector<cplx<T>> v((size_t)S::NTHR * N2);
  const int ncols = a.N * a.h;
  const int L = xf_num_tiles(a.stage);
  const T nan = std::numeric_limits<T>::quiet_NaN();
  for (int bx = 0; bx < ncols / S::W; ++bx) {
    auto issue = [&](int j) {
      if (j >= L) return;
      const XfTile t = xf_tile<N1, N2>(j, 0, a.stage);
      const cplx<T>* src = t.src == 0 ? a.dq : (t.src == 1 ? a.u0 : a.us);
      cplx<T>* dst = ring + (j % S::NSLOT) * S::SLOT;
      for (int r = 0; r < S::H; ++r)
        for (int c = 0; c < S::W; ++c) dst[r * S::W + c] = src[(t.row + r) * ncols + bx * S::W + c];
    };
    for (int e = 0; e < S::SM_ELEMS; ++e) sm[e] = cmake(nan, nan);
    for (int j = 0; j < S::NSLOT; ++j) issue(j);
    for (int t = 0; t < S::NTHR; ++t) xfused_twiddles<T, N1, N2>(a, tw, t, S::NTHR);
    for (auto& x : st)
      for (int q = 0; q < 3; ++q)
        for (int k = 0; k < N2; ++k) x.v[q][k] = czero<T>();
    for (int q = 0; q < 6; ++q) {
      for (int t = 0; t < S::NTHR; ++t) xfused_fwd1<T, N1, N2>(q, t, S::NTHR, ring, tw, X);
      for (int j = 3 * q; j < 3 * q + 3; ++j) issue(j + S::NSLOT);
      for (int t = 0; t < S::NTHR; ++t) xfused_fwd2<T, N1, N2>(a, bx, q, t, X, st[t]);
    }
    for (int t = 0; t < S::NTHR; ++t) xfused_leray<T, N1, N2>(a, bx, t, st[t]);
    for (int q = 0; q < 3; ++q) {
      const int cl = xf_comp_tiles(a.stage), j0 = 18 + q * cl;
      for (int t = 0; t < S::NTHR; ++t) {
        xfused_combine<T, N1, N2>(a, bx, 0, q, t, ring, st[t], &v[(size_t)t * N2]);
        xfused_inv1<T, N1, N2>(t, tw, X, &v[(size_t)t * N2]);
      }
      for (int j = j0; j < j0 + cl; ++j) issue(j + S::NSLOT);
      for (int t = 0; t < S::NTHR; ++t) xfused_inv2<T, N1, N2>(a, bx, 0, q, t, S::NTHR, X);
    }
    for (int t = 0; t < S::NTHR; ++t) xfused_clock<T, N1, N2>(a, bx, 0, t);
  }
}

template <typename T, int N1, int N2>
void run_xfused_prologue(const XFusedArgs<T>& a) {
  using S = XFusedShape<N1, N2>;
  std::vector<cplx<T>> sm(2 * S::P + S::W * S::LP);
  std::vector<cplx<T>> v((size_t)S::NTHR * N2);
  const int ncols = a.N * a.h;
  for (int bx = 0; bx < ncols / S::W; ++bx) {
    for (int t = 0; t < S::NTHR; ++t) xfused_twiddles<T, N1, N2>(a, sm.data(), t, S::NTHR);
    cplx<T>* X = sm.data() + 2 * S::P;
    for (int q = 0; q < 3; ++q) {
      for (int t = 0; t < S::NTHR; ++t) {
        xfused_prologue_load<T, N1, N2>(a, bx, 0, q, t, &v[(size_t)t * N2]);
        xfused_inv1<T, N1, N2>(t, sm.data(), X, &v[(size_t)t * N2]);
      }
      for (int t = 0; t < S::NTHR; ++t) xfused_inv2<T, N1, N2>(a, bx, 0, q, t, S::NTHR, X);
    }
  }
}

template <typename T>
bool fused_shape(const ns3d::Geom& g) {
  if (!g_use_fast || g.form != 0 || sizeof(T) != 4 || 3 * g.h != g.P) return false;
#define NS3D_HC_XS(A, B) \
  if (g.P == (A) * (B)) return true;
  NS3D_FOR_XFUSED(NS3D_HC_XS)
#undef NS3D_HC_XS
  return false;
}

// One stage with the fused x pass (W1 holds the x-inverse of `in` on entry,
// and of `out` on exit).
template <typename T>
void fused_stage(const ns3d::Geom& g, const SpecParams& sp, cplx<T>* u0, cplx<T>* us,
                 cplx<T>* out, int stage, std::vector<cplx<T>>& W1, std::vector<cplx<T>>& W2,
                 const std::vector<cplx<T>>& tw, Ns3dCtrl* ctrl, std::vector<cplx<T>>& sm) {
  using namespace ns3d;
  run_col<T, +1, true, true>(args_inv_y<T>(g, W1.data(), W2.data(), tw.data()), launch_inv_y(g, 1), sm);
  {
    ZArgs<T> za = args_z<T>(g, W2.data(), W1.data(), tw.data(), stage == 1 ? ctrl : nullptr);
    if (!run_z_fast_if_any<T>(za, g.P)) run_z<T>(za, launch_z(g, 1), sm);
  }
  run_col<T, -1, true, true>(args_fwd_y<T>(g, W1.data(), W2.data(), tw.data()), launch_fwd_y(g, 1), sm);
  if (stage == 1) step_dt_member(*ctrl, sp);
  XFusedArgs<T> x{};
  x.dq = W2.data();
  x.u0 = u0;
  x.us = us;
  x.out = out;
  x.ax = W1.data();
  x.tw = tw.data();
  std::vector<T> lam(3 * (g.h - 1) * (g.h - 1) + 1);
  {
    const SpecT<double> spd = spec_t<double>(sp);
    for (size_t k2 = 0; k2 < lam.size(); ++k2) lam[k2] = T(lambda_k<double>((int)k2, spd));
  }
  x.lam = lam.data();
  x.N = g.N;
  x.h = g.h;
  x.stage = stage;
  x.m6 = g.nDq;
  x.m3 = g.nU;
  x.mA = g.nA;
  x.sp = spec_t<T>(sp);
  x.ctrl = ctrl;
#define NS3D_HC_XF(A, B) \
  if (g.P == (A) * (B)) run_xfused<T, A, B>(x);
  NS3D_FOR_XFUSED(NS3D_HC_XF)
#undef NS3D_HC_XF
}

// rhs_stage for the advective and rotational forms (the plan's form path)
template <typename T>
void rhs_stage_form(const ns3d::Geom& g, const SpecParams& sp, const cplx<T>* in, cplx<T>* u0,
                    cplx<T>* us, cplx<T>* out, int stage, std::vector<cplx<T>>& W1,
                    std::vector<cplx<T>>& W2, const std::vector<cplx<T>>& tw, Ns3dCtrl* ctrl,
                    std::vector<cplx<T>>& sm) {
  using namespace ns3d;
  const long long N = g.N, P = g.P, h = g.h;
  const int nf = form_fields(g.form);
  for (long long i = 0; i < N * N * h; ++i)
    form_prep_point<T>(in, W1.data(), g.N, T(sp.kscale), g.form, i);
  Launch lx = launch_inv_x(g, 1);
  lx.gz = nf;
  run_col<T, +1, true, true>(args_inv_x<T>(g, W1.data(), W2.data(), tw.data()), lx, sm);
  Launch ly = launch_inv_y(g, 1);
  ly.gz = nf;
  run_col<T, +1, true, true>(args_inv_y<T>(g, W2.data(), W1.data(), tw.data()), ly, sm);
  ZArgs<T> az = args_z<T>(g, W1.data(), W2.data(), tw.data(), stage == 1 ? ctrl : nullptr);
  az.W = g.Wzf;
  az.ldw = g.ldwzf;
  az.in_bs = nf * P * P * h;
  az.out_bs = 3 * P * P * h;
  bool done = false;
  if (g_use_fast && g_form_W == 0 && sizeof(T) == 4 && g.form != 0 && 3 * g.h == g.P) {
#define NS3D_HC_ZR(A, B)                                            \
    if (g.P == (A) * (B)) {                                         \
      if (g.form == 2) run_zrot<T, A, B>(az, 1); else run_zadv<T, A, B>(az, 1); \
      done = true;                                                  \
    }
    NS3D_FOR_ZFAST(NS3D_HC_ZR)
#undef NS3D_HC_ZR
  }
  if (!done) run_zform<T>(az, g.form, Launch{cdiv(P, g.Wzf), g.P, 1, g.nthr_zf, g.smem_zf}, sm);
  Launch lfy = launch_fwd_y(g, 1);
  lfy.gz = 3;
  run_col<T, -1, true, true>(args_fwd_y<T>(g, W2.data(), W1.data(), tw.data()), lfy, sm);
  Launch lfx = launch_fwd_x(g, 1);
  lfx.gz = 3;
  run_col<T, -1, true, true>(args_fwd_x<T>(g, W1.data(), W2.data(), tw.data()), lfx, sm);
  SpecArgs<T> s{};
  s.bh = W2.data();
  s.u0 = (stage == 0) ? in : u0;
  s.us = us;
  s.out = out;
  s.N = g.N;
  s.h = g.h;
  s.nmem = 1;
  s.stage = stage;
  s.m6 = 3 * N * N * h;
  s.m3 = g.nU;
  s.sp = spec_t<T>(sp);
  s.ctrl = ctrl;
  s.form = g.form;
  if (stage == 1) step_dt_member(*ctrl, sp);
  for (int kx = 0; kx < g.N; ++kx)
    for (int j = 0; j < g.N * g.h; ++j) spectral_point<T>(s, 0, kx, j);
}

// One evaluation of Algorithm 2 and the spectral step on member 0.
template <typename T>
void rhs_stage(const ns3d::Geom& g, const SpecParams& sp, const cplx<T>* in, cplx<T>* u0,
               cplx<T>* us, cplx<T>* out, int stage, std::vector<cplx<T>>& W1,
               std::vector<cplx<T>>& W2, const std::vector<cplx<T>>& tw, Ns3dCtrl* ctrl,
               std::vector<cplx<T>>& sm) {
  using namespace ns3d;
  if (g.form != 0) {
    rhs_stage_form<T>(g, sp, in, u0, us, out, stage, W1, W2, tw, ctrl, sm);
    return;
  }
  run_col<T, +1, true, true>(args_inv_x<T>(g, in, W1.data(), tw.data()), launch_inv_x(g, 1), sm);
  run_col<T, +1, true, true>(args_inv_y<T>(g, W1.data(), W2.data(), tw.data()), launch_inv_y(g, 1), sm);
  {
    ZArgs<T> za = args_z<T>(g, W2.data(), W1.data(), tw.data(), stage == 1 ? ctrl : nullptr);
    if (!(g_use_fast && run_z_fast_if_any<T>(za, g.P))) run_z<T>(za, launch_z(g, 1), sm);
  }
  run_col<T, -1, true, true>(args_fwd_y<T>(g, W1.data(), W2.data(), tw.data()), launch_fwd_y(g, 1), sm);
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
  s.sp = spec_t<T>(sp);
  s.ctrl = ctrl;
  if (stage == 1) step_dt_member(*ctrl, sp);
  for (int kx = 0; kx < g.N; ++kx)
    for (int j = 0; j < g.N * g.h; ++j) spectral_point<T>(s, 0, kx, j);
}

template <typename T>
int run(int N, int P, const double* prm, const void* uin, void* uout, int nsteps, double dt,
        double* t_out) {
  ns3d::Geom g;
  if (!ns3d::make_geom(N, P, (int)sizeof(cplx<T>), &g) || !ns3d::set_form_geom(&g, g_form)) return 1;
  if (g_form_W > 0 && g.form != 0) {
    bool found = false;
    for (const ns3d::FormTile& t : ns3d::form_tile_candidates(g))
      if (t.W == g_form_W && !found) {
        ns3d::set_form_tile(&g, t);
        found = true;
      }
    if (!found) return 1;
  }
  // prm: L nu s theta eps0 mN_coef q_form cfl
  SpecParams sp = ns3d::make_spec_params(N, P, prm[0], prm[1], prm[2], prm[3], prm[4], prm[5],
                                         (int)prm[6], prm[7], dt);
  std::vector<cplx<T>> tw = ns3d::make_twiddles<T>(P);
  std::vector<cplx<T>> U0(g.nU), US(g.nU), W1(g.nW1), W2(g.nW2);
  size_t sm_elems = std::max(std::max(g.smem_c, g.smem_z), g.smem_zf) / sizeof(cplx<T>) + 16;
  std::vector<cplx<T>> sm(sm_elems);
  d1_to_compact((const cplx<T>*)uin, U0.data(), N);
  Ns3dCtrl ctrl{};
  if (nsteps == 0) {
    rhs_stage<T>(g, sp, U0.data(), nullptr, nullptr, US.data(), 0, W1, W2, tw, &ctrl, sm);
    compact_to_d1(US.data(), (cplx<T>*)uout, N);
    return 0;
  }
  if (fused_shape<T>(g)) {
    XFusedArgs<T> pa{};
    pa.u0 = U0.data();
    pa.ax = W1.data();
    pa.tw = tw.data();
    pa.N = g.N;
    pa.h = g.h;
    pa.m3 = g.nU;
    pa.mA = g.nA;
#define NS3D_HC_XP(A, B) \
    if (g.P == (A) * (B)) run_xfused_prologue<T, A, B>(pa);
    NS3D_FOR_XFUSED(NS3D_HC_XP)
#undef NS3D_HC_XP
    for (int n = 0; n < nsteps; ++n) {
      fused_stage<T>(g, sp, U0.data(), US.data(), US.data(), 1, W1, W2, tw, &ctrl, sm);
      fused_stage<T>(g, sp, U0.data(), US.data(), US.data(), 2, W1, W2, tw, &ctrl, sm);
      fused_stage<T>(g, sp, U0.data(), US.data(), U0.data(), 3, W1, W2, tw, &ctrl, sm);
    }
  } else {
    for (int n = 0; n < nsteps; ++n) {
      rhs_stage<T>(g, sp, U0.data(), U0.data(), US.data(), US.data(), 1, W1, W2, tw, &ctrl, sm);
      rhs_stage<T>(g, sp, US.data(), U0.data(), US.data(), US.data(), 2, W1, W2, tw, &ctrl, sm);
      rhs_stage<T>(g, sp, US.data(), U0.data(), US.data(), U0.data(), 3, W1, W2, tw, &ctrl, sm);
    }
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

// 0: emulate the generic tile z pass even where a register-resident one exists.
void ns3d_hostcheck_use_fast(int mode) { g_use_fast = mode; }

// nonlinear form of later ns3d_hostcheck_run calls (0, 1 or 2)
void ns3d_hostcheck_set_form(int form) { g_form = form; }

// zform tile width of later form-1/2 runs (0: the default shape)
void ns3d_hostcheck_set_form_tile(int W) { g_form_W = W; }

// One column pass of the three-pass kernel at P = 1536 (N = 1024) on a
// [rows][ncols] array: sign > 0 the padded inverse (N rows in, P out),
// sign < 0 the truncated forward (P rows in, N out, Nyquist row zero).
int ns3d_hostcheck_colpass3(int sign, const void* in, void* out, int ncols) {
  constexpr int P = 16 * 12 * 8, N = 2 * P / 3, h = N / 2;
  const std::vector<cplx<float>> tw = ns3d::make_twiddles<float>(P);
  ColArgs<float> a{};
  a.in = static_cast<const cplx<float>*>(in);
  a.out = static_cast<cplx<float>*>(out);
  a.tw = tw.data();
  a.pl.n = P;
  a.h = h;
  a.ncols = ncols;
  a.in_cs = a.out_cs = 1;
  a.in_rs = a.out_rs = ncols;
  a.scale = 1.0f;
  if (sign > 0) {
    a.nrow_in = N; a.nrow_out = P; a.pad_in = 1; a.trunc_out = 0;
    run_colfast3<float, +1, 16, 12, 8>(a, 1, 1);
  } else {
    a.nrow_in = P; a.nrow_out = N; a.pad_in = 0; a.trunc_out = 1;
    run_colfast3<float, -1, 16, 12, 8>(a, 1, 1);
  }
  return 0;
}

// The three-pass z pass at P = 1536 on rows x < nx of Bq-like input
// [3][nx][P][h] -> Cq-like output [6][nx][P][h]; returns the status flags and
// the CFL maximum.
int ns3d_hostcheck_zpass3(const void* in, void* out, int nx, double* umax) {
  constexpr int P = 1536, h = P / 3;
  const std::vector<cplx<float>> tw = ns3d::make_twiddles<float>(P);
  Ns3dCtrl ctrl{};
  ZArgs<float> a{};
  a.in = static_cast<const cplx<float>*>(in);
  a.out = static_cast<cplx<float>*>(out);
  a.tw = tw.data();
  a.P = P;
  a.h = h;
  a.in_cs = a.out_cs = (long long)nx * P * h;
  a.xs = (long long)P * h;
  a.ctrl = &ctrl;
#define NS3D_HC_Z3(A, B, C) run_zfast3<float, A, B, C>(a, 1, nx);
  NS3D_FOR_ZFAST3(NS3D_HC_Z3)
#undef NS3D_HC_Z3
  std::memcpy(umax, &ctrl.umax_bits, sizeof(double));
  return ctrl.status;
}

// The FP64 three-pass z pass (double-single arithmetic) at a padded size P of
// NS3D_FOR_ZFAST3_F64 on rows x < nx of a [3][nx][P][h] complex128 array into
// [6][nx][P][h]; returns the status flags (-1: no kernel at P) and the CFL
// maximum.
int ns3d_hostcheck_zpass3_f64(int P, const void* in, void* out, int nx, double* umax) {
  const int h = P / 3;
  const std::vector<cplx<double>> tw = ns3d::make_twiddles<double>(P);
  Ns3dCtrl ctrl{};
  ZArgs<double> a{};
  a.in = static_cast<const cplx<double>*>(in);
  a.out = static_cast<cplx<double>*>(out);
  a.tw = tw.data();
  a.P = P;
  a.h = h;
  a.in_cs = a.out_cs = (long long)nx * P * h;
  a.xs = (long long)P * h;
  a.ctrl = &ctrl;
  bool done = false;
#define NS3D_HC_Z3D(A, B, C)                 \
  if (P == (A) * (B) * (C)) {                \
    run_zfast3<double, A, B, C>(a, 1, nx);   \
    done = true;                             \
  }
  NS3D_FOR_ZFAST3_F64(NS3D_HC_Z3D)
#undef NS3D_HC_Z3D
  if (!done) return -1;
  std::memcpy(umax, &ctrl.umax_bits, sizeof(double));
  return ctrl.status;
}

// The adjoint z pass on x rows < nx of a [9][P][P][h] complex64 array: the
// register-resident kernel into out_fast and the generic tile block into
// out_generic (both [3][P][P][h]).  P must be a register size (48, 96, 192,
// 384); returns -1 otherwise.
int ns3d_hostcheck_zadj(int P, const void* in, void* out_fast, void* out_generic, int nx) {
  const int h = P / 3;
  const std::vector<cplx<float>> tw = ns3d::make_twiddles<float>(P);
  ZArgs<float> a{};
  a.in = static_cast<const cplx<float>*>(in);
  a.out = static_cast<cplx<float>*>(out_fast);
  a.tw = tw.data();
  a.P = P;
  a.h = h;
  a.in_cs = a.out_cs = (long long)P * P * h;
  a.xs = (long long)P * h;
  bool done = false;
#define NS3D_HC_ZA(A, B)              \
  if (P == (A) * (B)) {               \
    run_zadjf<float, A, B>(a, nx);    \
    done = true;                      \
  }
  NS3D_FOR_ZFAST(NS3D_HC_ZA)
#undef NS3D_HC_ZA
  if (!done) return -1;
  ZAdjArgs<float> g{};
  g.in = static_cast<const cplx<float>*>(in);
  g.out = static_cast<cplx<float>*>(out_generic);
  g.tw = tw.data();
  if (!ns3d::make_fft_plan(P, &g.pl)) return -1;
  g.P = P;
  g.h = h;
  g.W = 8;
  g.ldw = 9;
  std::vector<cplx<float>> sm((size_t)7 * P * g.ldw);
  for (int by = 0; by < nx; ++by)
    for (int bx = 0; bx < (P + g.W - 1) / g.W; ++bx) zadj_block<float>(g, bx, by, 0, 1, sm.data(), HostSync{});
  return 0;
}

// Radix plan chosen for length n (for tests).
int ns3d_hostcheck_plan(int n, int* radix, int maxp) {
  FftPlanDev pl;
  if (!ns3d::make_fft_plan(n, &pl)) return -1;
  for (int i = 0; i < pl.npass && i < maxp; ++i) radix[i] = pl.radix[i];
  return pl.npass;
}
}
