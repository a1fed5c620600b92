// Fused x pass (FP32, P = N1 * N2 at the default padding P = 3N/2): the
// forward x transform of the six products with truncation, the spectral step
// and SSP-RK3 combine (section 2.3, eq. RK3), and the inverse x transform with
// padding of the new stage state, for a tile of W (ky, kz) columns.
//
//   inputs are staged in shared memory as tiles of H = N/2 rows x W columns
//     (a ring of NSLOT slots, filled by the tensor memory accelerator on the
//     GPU): each product component takes 3 tiles (P = 3H rows of Dq), each
//     state component 2 (N = 2H rows of u_n, and of the stage state at stages
//     2 and 3)
//   forward, per product component: pass 1 radix N1 (staged tile -> twiddle
//     -> X), pass 2 radix N2: thread (column, k1) receives B_hat at the
//     positions p = k1 + N1 k2 and accumulates b_hat_j = -i kappa_l B_hat_jl in
//     registers
//   Leray projection and lambda_k in registers at those positions; then per
//     state component the RK3 combine (the new state is stored: it is the
//     next stage's state) and the inverse transform with the transposed
//     factorisation P = N2 * N1: its first pass (radix N2 over positions
//     k1 + N1 k2) works on the thread's registers, its second (radix N1)
//     writes the x-inverse array A of the next stage.
//
// This replaces the forward-x, spectral and (next stage) inverse-x kernels and
// their B_hat round trip through memory.  Phases are separate functions with
// an explicit per-thread state so that the CPU emulator can run them thread by
// thread; the staging (which rows of which array go to which slot) is one
// function shared by both.
#pragma once

#include "ns3d_colfast.cuh"

#define NS3D_FOR_XFUSED(X) X(24, 16) X(12, 16) X(12, 8) X(6, 8)

// (ky, kz) columns per CTA; also the width of the TMA boxes (xfused_maps.cu)
constexpr int kXfusedW = 8;

template <int N1, int N2>
struct XFusedShape {
  static constexpr int P = N1 * N2;
  static constexpr int H = P / 3;         // N / 2: rows of one staged tile
  static constexpr int W = kXfusedW;
  static constexpr int NTHR = W * N1;     // one pass-2 task (column, k1) per thread
  static constexpr int LP = P + 1;
  static constexpr int NSLOT = 9;         // staging ring: three product components
  static constexpr int SLOT = H * W;      // elements of one staged tile
  // shared memory (complex elements): ring | twiddles (forward, inverse) | X
  static constexpr int OFF_TW = NSLOT * SLOT;
  static constexpr int OFF_X = OFF_TW + 2 * P;
  static constexpr int SM_ELEMS = OFF_X + W * LP;
};

template <typename T>
struct XFusedArgs {
  const cplx<T>* dq;   // Dq [m][6][x P][ky N][kz h]
  const cplx<T>* u0;   // state at t_n           [m][3][N][N][h]
  const cplx<T>* us;   // stage state (stages 2, 3)
  cplx<T>* out;        // new stage state
  cplx<T>* ax;         // A of the new state     [m][3][x P][ky N][kz h]
  const cplx<T>* tw;   // exp(-2 pi i e / P)
  const T* lam;        // lambda_k by |k|^2 (integer), 0 .. 3 (h - 1)^2
  int N, h, stage;
  unsigned extra_tx;   // 0; a test of the timeout path expects more bytes on tile 0
  long long m6, m3, mA;   // member strides of Dq, U, A
  SpecT<T> sp;
  Ns3dCtrl* ctrl;
};

template <typename T, int N1, int N2>
struct XFusedState {
  cplx<T> v[3][N2];   // b_hat, then the projected b_hat, at positions k1 + N1 k2
  T lam[N2];          // lambda_k at those positions
};

// ---------------------------------------------------------------- staging
// Tiles of one stage, in consumption order: product components q = 0..5 (3
// row blocks of H each), then per state component q = 0..2 the 2 row blocks
// of u_n and, at stages 2 and 3, the 2 of the stage state.  Tile j goes to
// slot j % NSLOT once tile j - NSLOT has been consumed.
NS3D_HDC int xf_comp_tiles(int stage) { return stage == 1 ? 2 : 4; }
NS3D_HDC int xf_num_tiles(int stage) { return 18 + 3 * xf_comp_tiles(stage); }

struct XfTile {
  int src;         // 0 Dq, 1 u_n, 2 stage state
  long long row;   // first row in the array viewed as [rows][N h] over all members
};

template <int N1, int N2>
NS3D_HD XfTile xf_tile(int j, int m, int stage) {
  using S = XFusedShape<N1, N2>;
  XfTile t;
  if (j < 18) {
    t.src = 0;
    t.row = (long long)(m * 6 + j / 3) * S::P + (j % 3) * S::H;
    return t;
  }
  const int cl = xf_comp_tiles(stage);
  const int q = (j - 18) / cl, r = (j - 18) % cl;
  t.src = 1 + r / 2;
  t.row = (long long)(m * 3 + q) * (2 * S::H) + (r % 2) * S::H;
  return t;
}

// ---------------------------------------------------------------- phases

template <typename T, int N1, int N2>
NS3D_HD void xfused_twiddles(const XFusedArgs<T>& a, cplx<T>* tw, int tid, int nthr) {
  using S = XFusedShape<N1, N2>;
  for (int e = tid; e < S::P; e += nthr) {
    const cplx<T> w = a.tw[e];
    tw[e] = w;                          // forward
    tw[S::P + e] = cmake(w.x, -w.y);    // inverse
  }
}

// signed frequency of transform position p in the retained band, or a value
// outside [-h+1, h-1] when p lies in the dropped band or is the Nyquist row
template <int P, int H>
NS3D_HD int xf_freq(int p) {
  return p < H ? p : (p > P - H ? p - P : (1 << 20));
}

// Signed frequency of position p = k1 + N1 k2 (k2 a compile-time block
// index): p in a PAD_LOW block, p - P in a PAD_HIGH block, decided per
// position in a PAD_MIXED block (out of band in a PAD_ZERO block).
template <int N1, int N2>
NS3D_HD int xf_sx(int k1, int k2) {
  using S = XFusedShape<N1, N2>;
  const int reg = pad_region(N1 * k2, N1, S::P, S::H);
  const int p = k1 + N1 * k2;
  return reg == PAD_LOW ? p : (reg == PAD_HIGH ? p - S::P : xf_freq<S::P, S::H>(p));
}

// forward pass 1 of product component q (its three staged tiles are
// consecutive slots: P rows of W columns)
template <typename T, int N1, int N2>
NS3D_HD void xfused_fwd1(int q, int tid, int nthr, const cplx<T>* ring, const cplx<T>* tw,
                         cplx<T>* X) {
  using S = XFusedShape<N1, N2>;
  const cplx<T>* tile = ring + 3 * (q % 3) * S::SLOT;
  for (int t = tid; t < S::W * N2; t += nthr) {
    const int col = t % S::W, j2 = t / S::W;
    cplx<T> v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) v[j1] = tile[(N2 * j1 + j2) * S::W + col];
    Dft<N1, -1>::run(v);
    cplx<T>* D = X + col * S::LP + j2 * N1;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) D[k1] = k1 == 0 ? v[k1] : v[k1] * tw[j2 * k1];   // tw[0] = 1
  }
}

// b_r += -i kappa_s B, b_s += -i kappa_r B (r != s) for component (r, s)
template <typename T, int N1, int N2, int R, int S_>
NS3D_HD void xf_accumulate(const cplx<T>* v, const T* kx, T kyv, T kzv,
                           XFusedState<T, N1, N2>& st) {
  using S = XFusedShape<N1, N2>;
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    if (pad_region(N1 * k2, N1, S::P, S::H) == PAD_ZERO) continue;
    const T kap[3] = {kx[k2], kyv, kzv};
    const cplx<T> mb = cmake(v[k2].y, -v[k2].x);   // -i B
    st.v[R][k2] = st.v[R][k2] + kap[S_] * mb;
    if (R != S_) st.v[S_][k2] = st.v[S_][k2] + kap[R] * mb;
  }
}

// forward pass 2 of component q and accumulation of b_hat (unnormalised)
template <typename T, int N1, int N2>
NS3D_HD void xfused_fwd2(const XFusedArgs<T>& a, int bx, int q, int tid, const cplx<T>* X,
                         XFusedState<T, N1, N2>& st) {
  using S = XFusedShape<N1, N2>;
  const int col = tid % S::W, k1 = tid / S::W;
  const int c = bx * S::W + col;
  const int h = a.h, N = a.N;
  const int ky = (c / h) % N, kz = c % h;
  const T ks = a.sp.kscale;
  const T kyv = ks * T(ky < h ? ky : ky - N), kzv = ks * T(kz);
  T kx[N2];
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) kx[k2] = ks * T(xf_sx<N1, N2>(k1, k2));
  cplx<T> v[N2];
  const cplx<T>* D = X + col * S::LP + k1;
#pragma unroll
  for (int j = 0; j < N2; ++j) v[j] = D[j * N1];
  Dft<N2, -1>::run(v);
  // components of B in the order 00 01 02 11 12 22
  switch (q) {
    case 0: xf_accumulate<T, N1, N2, 0, 0>(v, kx, kyv, kzv, st); break;
    case 1: xf_accumulate<T, N1, N2, 0, 1>(v, kx, kyv, kzv, st); break;
    case 2: xf_accumulate<T, N1, N2, 0, 2>(v, kx, kyv, kzv, st); break;
    case 3: xf_accumulate<T, N1, N2, 1, 1>(v, kx, kyv, kzv, st); break;
    case 4: xf_accumulate<T, N1, N2, 1, 2>(v, kx, kyv, kzv, st); break;
    default: xf_accumulate<T, N1, N2, 2, 2>(v, kx, kyv, kzv, st); break;
  }
}

// Leray projection of the normalised b_hat and lambda_k, in registers;
// positions outside the retained band (and k = 0) get zero
template <typename T, int N1, int N2>
NS3D_HD void xfused_leray(const XFusedArgs<T>& a, int bx, int tid, XFusedState<T, N1, N2>& st) {
  using S = XFusedShape<N1, N2>;
  const int col = tid % S::W, k1 = tid / S::W;
  const int h = a.h, N = a.N;
  const int c = bx * S::W + col;
  const int ky = (c / h) % N, kz = c % h;
  const int sy = ky < h ? ky : ky - N;
  const SpecT<T>& sp = a.sp;
  const T kyv = sp.kscale * T(sy), kzv = sp.kscale * T(kz);
  const int kyz2 = sy * sy + kz * kz;
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int reg = pad_region(N1 * k2, N1, S::P, S::H);
    const int sx = xf_sx<N1, N2>(k1, k2);
    const int k2i = sx * sx + kyz2;
    const bool band = reg == PAD_LOW || reg == PAD_HIGH || (reg == PAD_MIXED && sx > -h && sx < h);
    const bool live = band && ky != h && k2i > 0;
    cplx<T> b0 = czero<T>(), b1 = czero<T>(), b2 = czero<T>();
    T lam = T(0);
    if (live) {
      const T kxv = sp.kscale * T(sx);
      b0 = sp.inv_P3 * st.v[0][k2];
      b1 = sp.inv_P3 * st.v[1][k2];
      b2 = sp.inv_P3 * st.v[2][k2];
      const T kap2 = kxv * kxv + kyv * kyv + kzv * kzv;
      const cplx<T> kb = (T(1) / kap2) * (kxv * b0 + kyv * b1 + kzv * b2);
      b0 = b0 - kxv * kb;
      b1 = b1 - kyv * kb;
      b2 = b2 - kzv * kb;
      lam = a.lam[k2i];
    }
    st.v[0][k2] = b0;
    st.v[1][k2] = b1;
    st.v[2][k2] = b2;
    st.lam[k2] = lam;
  }
}

// RK3 combine of state component q (its staged tiles from the ring), store
// of the new state; v receives the new state at the thread's positions
template <typename T, int N1, int N2>
NS3D_HD void xfused_combine(const XFusedArgs<T>& a, int bx, int m, int q, int tid,
                            const cplx<T>* ring, const XFusedState<T, N1, N2>& st, cplx<T>* v) {
  using S = XFusedShape<N1, N2>;
  const int col = tid % S::W, k1 = tid / S::W;
  const int h = a.h, N = a.N;
  const int ncols = N * h;
  const int c = bx * S::W + col;
  const bool nyq = (c / h) % N == h;   // the Nyquist column ky = h stays zero
  const long long plane = (long long)N * ncols;
  const Ns3dCtrl& cc = a.ctrl[m];
  const T dt = ctrl_dt<T>(cc);
  const bool frozen = !(dt > T(0));
  const int j0 = 18 + q * xf_comp_tiles(a.stage);   // tiles of u_n's component q
  // rows kx < H and kx >= H of u_n and of the stage state
  const cplx<T>* u0lo = ring + (j0 % S::NSLOT) * S::SLOT + col;
  const cplx<T>* u0hi = ring + ((j0 + 1) % S::NSLOT) * S::SLOT + col;
  const cplx<T>* uslo = ring + ((j0 + 2) % S::NSLOT) * S::SLOT + col;
  const cplx<T>* ushi = ring + ((j0 + 3) % S::NSLOT) * S::SLOT + col;
  cplx<T>* o = a.out + m * a.m3 + q * plane + c;
  const bool store = !(frozen && a.out == a.u0);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int reg = pad_region(N1 * k2, N1, S::P, S::H);
    cplx<T> nv = czero<T>();
    if (reg != PAD_ZERO) {
      const int sx = xf_sx<N1, N2>(k1, k2);
      const bool band = reg != PAD_MIXED || (sx > -h && sx < h);
      // row kx of the N-row arrays: p (low block), p - H (high block)
      const int kx = sx < 0 ? sx + N : sx;
      const int half = reg == PAD_LOW ? 0 : (reg == PAD_HIGH ? 1 : (kx >= S::H ? 1 : 0));
      const int r = (kx - half * S::H) * S::W;
      if (band) {
        if (!nyq) {
          const cplx<T> u0 = (half ? u0hi : u0lo)[r];
          if (frozen) {
            nv = u0;
          } else {
            const cplx<T> pb = q == 0 ? st.v[0][k2] : (q == 1 ? st.v[1][k2] : st.v[2][k2]);
            if (a.stage == 1) {
              nv = u0 + dt * (pb - st.lam[k2] * u0);
            } else {
              const cplx<T> us = (half ? ushi : uslo)[r];
              const cplx<T> w = us + dt * (pb - st.lam[k2] * us);
              nv = a.stage == 2 ? T(0.75) * u0 + T(0.25) * w
                                : T(1.0 / 3.0) * u0 + T(2.0 / 3.0) * w;
            }
          }
        }
        if (store) o[(long long)kx * ncols] = nv;
      }
    }
    v[k2] = nv;
  }
}

// Prologue (the x-inverse of a state set outside a step): the stored state
// of component q at the thread's positions, exactly the values the combine
// leaves in v for a member that does not move, so that xfused_inv1/2 on them
// give A bit for bit as the fused pass would
template <typename T, int N1, int N2>
NS3D_HD void xfused_prologue_load(const XFusedArgs<T>& a, int bx, int m, int q, int tid,
                                  cplx<T>* v) {
  using S = XFusedShape<N1, N2>;
  const int col = tid % S::W, k1 = tid / S::W;
  const int h = a.h, N = a.N;
  const int ncols = N * h;
  const int c = bx * S::W + col;
  const bool nyq = (c / h) % N == h;
  const cplx<T>* u = a.u0 + m * a.m3 + (long long)q * N * ncols + c;
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const int sx = xf_freq<S::P, S::H>(k1 + N1 * k2);
    cplx<T> nv = czero<T>();
    if (sx > -h && sx < h && !nyq) nv = u[(long long)(sx < 0 ? sx + N : sx) * ncols];
    v[k2] = nv;
  }
}

// the thread holding k = 0 of the member advances its clock after stage 3
// (the other threads of this launch read only dt)
template <typename T, int N1, int N2>
NS3D_HD void xfused_clock(const XFusedArgs<T>& a, int bx, int m, int tid) {
  using S = XFusedShape<N1, N2>;
  if (a.stage != 3 || bx != 0 || tid != 0) return;
  Ns3dCtrl& cc = a.ctrl[m];
  if (ctrl_dt<T>(cc) > T(0)) {
    cc.t += cc.dt;
    cc.nsteps += 1;
  }
  cc.umax_bits = 0ull;
  (void)sizeof(S);
}

// inverse pass 1: radix N2 over the thread's positions k1 + N1 k2, twiddle,
// to X
template <typename T, int N1, int N2>
NS3D_HD void xfused_inv1(int tid, const cplx<T>* tw, cplx<T>* X, cplx<T>* v) {
  using S = XFusedShape<N1, N2>;
  const int col = tid % S::W, k1 = tid / S::W;
  Dft<N2, +1>::run(v);
  const cplx<T>* twi = tw + S::P;
  cplx<T>* D = X + col * S::LP + k1 * N2;
#pragma unroll
  for (int k = 0; k < N2; ++k) D[k] = k == 0 ? v[k] : v[k] * twi[k1 * k];   // twi[0] = 1
}

// inverse pass 2 of component q: radix N1, rows x = kappa + N2 k of A
template <typename T, int N1, int N2>
NS3D_HD void xfused_inv2(const XFusedArgs<T>& a, int bx, int m, int q, int tid, int nthr,
                         const cplx<T>* X) {
  using S = XFusedShape<N1, N2>;
  const int ncols = a.N * a.h;
  const int c0 = bx * S::W;
  cplx<T>* A = a.ax + m * a.mA + (long long)q * S::P * ncols + c0;
  for (int t = tid; t < S::W * N2; t += nthr) {
    const int col = t % S::W, kap = t / S::W;
    cplx<T> v[N1];
    const cplx<T>* D = X + col * S::LP + kap;
#pragma unroll
    for (int j = 0; j < N1; ++j) v[j] = D[j * N2];
    Dft<N1, +1>::run(v);
#pragma unroll
    for (int k = 0; k < N1; ++k) A[(kap + N2 * k) * ncols + col] = v[k];
  }
}
