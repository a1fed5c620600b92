// Fused z pass with register-resident transforms, for padded sizes
// P = N1 * N2 with both radices in registers (P = 48, 96, 192, 384).
//
// Same arithmetic as zfused_block (Algorithm 2 steps 2-4 along z: c2r of the
// three velocity components with the kz padding, the six products, the CFL
// maximum, r2c truncated to kz < N/2), organised so that each transform makes
// a single trip through shared memory:
//
//   inverse, pass 1   radix N1 over positions N2*j1 + j2 (task j2), read from
//                     global memory with the padding, twiddled, to shared memory
//   inverse, pass 2   radix N2 (task k1): thread (pair g, k1) keeps the physical
//                     values at positions k1 + N1*k2, k2 < N2, in registers
//   forward, pass 1   radix N2 over the SAME positions (the forward transform
//                     uses the transposed factorisation P = N2 * N1), products
//                     formed in registers, twiddled, to shared memory
//   forward, pass 2   radix N1, in place in shared memory
//   extraction        two real lines from one complex line, truncated, stored
//
// A CTA holds NPAIR pairs of adjacent y columns; a pair's three inverse lines
// are u0+iu1 of each column and u2(c)+iu2(c'), its six forward lines are
// B00+iB01, B02+iB11, B12+iB22 of each column, done three per round.
//
// The kernel body is a sequence of phase functions separated by block
// barriers; per-thread state is an explicit struct, so the CPU emulator can run
// the phases thread by thread (hostcheck.cpp).
#pragma once

#include "ns3d_blocks.cuh"

// Padded sizes with a register-resident z pass (FP32): P = N1 * N2, used with
// the default padding h = N/2 = P/3 (compile-time zero band).
#define NS3D_FOR_ZFAST(X) X(24, 16) X(12, 16) X(12, 8) X(6, 8)

template <typename T, int N1, int N2>
struct ZFastState {
  cplx<T> z[3][N2];   // inverse results of the pair at positions k1 + N1 k2
  T umax;             // max of |u0| + |u1| + |u2| over the thread's points
  int bad;
};

template <int N1, int N2>
struct ZFastShape {
  static constexpr int P = N1 * N2;
  static constexpr int H = P / 3;                     // N/2 of the default padding P = 3N/2
  // pairs per CTA: 96-thread blocks where N2 = 16 (four blocks of 3 warps per SM
  // beat two of 6 at the same residency), else 16
  static constexpr int NPAIR = N2 == 16 ? 96 / N1 : 16;
  static constexpr int NTHR = NPAIR * N1;
  static constexpr int Y = 2 * NPAIR;                 // columns per CTA
  // Exchange rows are padded by one element so that the strided pass stores
  // (stride N1 + 1 or N2 + 1 across threads) hit distinct shared-memory banks,
  // and lines start 8 elements (mod 16) apart, so that where a half-warp spans
  // two lines (N2 = 8: inverse pass 1 and forward pass 2) their rows fall in
  // the other half of the banks.
  static constexpr int LP0 = P + (N1 > N2 ? N1 : N2);
  static constexpr int LP = LP0 + (24 - LP0 % 16) % 16;
  // blocks per SM the registers are capped for: 12 warps at N2 = 16 (the
  // 168-register state), 18 warps at N2 = 8 (a 2 x 8 complex state per line)
  static constexpr int MINB = N2 == 16 ? 4 : 3;
  // shared memory in complex elements: two twiddle tables + exchange [NPAIR][3][LP]
  // (followed by NTHR reduction slots of T)
  static constexpr int SM_ELEMS = 2 * P + NPAIR * 3 * LP;
};

template <typename T, int N1, int N2>
struct ZFastCtx {
  const ZArgs<T>* a;
  int bx, by, bz;
  int y0, ncol;
  cplx<T>* twi;  // twi[k1 * N2 + j2] = exp(+2 pi i j2 k1 / P)  (inverse pass 1)
  cplx<T>* twf;  // twf[k * N1 + k1] = exp(-2 pi i k1 k / P)    (forward pass 1)
  cplx<T>* X;    // shared exchange buffer
};

// forward-pass exchange: natural position p = kappa + N2 k of a line
template <int N1, int N2>
NS3D_HD int zfast_fpos(int p) {
  return (p / N2) * (N2 + 1) + p % N2;
}

template <typename T, int N1, int N2>
NS3D_HD ZFastCtx<T, N1, N2> zfast_ctx(const ZArgs<T>& a, int bx, int by, int bz, cplx<T>* sm) {
  using S = ZFastShape<N1, N2>;
  ZFastCtx<T, N1, N2> c;
  c.a = &a;
  c.bx = bx;
  c.by = by;
  c.bz = bz;
  c.y0 = bx * S::Y;
  c.ncol = imin(S::Y, S::P - c.y0);
  c.twi = sm;
  c.twf = sm + S::P;
  c.X = sm + 2 * S::P;
  return c;
}

template <typename T, int N1, int N2>
NS3D_HD void zfast_load_twiddles(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  for (int e = tid; e < N1 * N2; e += nthr) {
    const int k1 = e / N2, j2 = e % N2;      // twi layout
    cplx<T> w = c.a->tw[j2 * k1];
    w.y = -w.y;
    c.twi[e] = w;
    const int k = e / N1, kk = e % N1;       // twf layout
    c.twf[e] = c.a->tw[kk * k];
  }
}

// inverse pass 1, task t = (pair g, line l, j2), j2 fastest for coalesced
// loads: the N1 inputs of the task from global memory (padding band known at
// compile time) ...
template <typename T, int N1, int N2>
NS3D_HD void zfast_inv1_load(const ZFastCtx<T, N1, N2>& c, int t, cplx<T>* v) {
  using S = ZFastShape<N1, N2>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  const cplx<T>* in = a.in + c.bz * a.in_bs + c.by * a.xs + (long long)c.y0 * h;
  const int j2 = t % N2;
  const int l = (t / N2) % 3;
  const int g = t / (3 * N2);
  const int ca = 2 * g + (l == 1 ? 1 : 0);
  const int cb = 2 * g + (l == 0 ? 0 : 1);
  const cplx<T>* ia = in + (l == 2 ? 2 : 0) * a.in_cs;
  const cplx<T>* ib = in + (l == 2 ? 2 : 1) * a.in_cs;
  const bool full = (S::P % S::Y == 0);     // every tile has Y columns
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) {
    // positions N2 j1 .. N2 j1 + N2 - 1: the zero band is known at compile time
    const int p = N2 * j1 + j2;
    const int reg = pad_region(N2 * j1, N2, S::P, S::H);
    if (reg == PAD_ZERO) {
      v[j1] = czero<T>();
    } else if (full && reg == PAD_LOW) {          // u_a[p] + i u_b[p]
      cplx<T> x = ia[ca * h + p], y = ib[cb * h + p];
      if (j1 == 0 && p == 0) {
        x.y = T(0);
        y.y = T(0);
      }
      v[j1] = cmake(x.x - y.y, x.y + y.x);
    } else if (full && reg == PAD_HIGH) {         // conj(u_a[P-p]) + i conj(u_b[P-p])
      const cplx<T> x = ia[ca * h + (S::P - p)], y = ib[cb * h + (S::P - p)];
      v[j1] = cmake(x.x + y.y, -x.y + y.x);
    } else {
      v[j1] = pack2(ia, ib, S::P, S::H, p, ca, cb, c.ncol);
    }
  }
}

// ... and its radix-N1 DFT, twiddle and store to the exchange buffer
template <typename T, int N1, int N2>
NS3D_HD void zfast_inv1_finish(const ZFastCtx<T, N1, N2>& c, int t, cplx<T>* v) {
  using S = ZFastShape<N1, N2>;
  const int j2 = t % N2;
  const int l = (t / N2) % 3;
  const int g = t / (3 * N2);
  Dft<N1, +1>::run(v);
  cplx<T>* X = c.X + (g * 3 + l) * S::LP;
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1)
    X[j2 * (N1 + 1) + k1] = k1 == 0 ? v[k1] : v[k1] * c.twi[k1 * N2 + j2];   // twi[k1 N2] = 1
}

// inverse pass 1: each thread takes tasks t and t + nthr at a time and issues
// the global loads of both before either transform, so that one task's load
// latency overlaps the other's (the task count is a multiple of 2 nthr)
template <typename T, int N1, int N2>
NS3D_HD void zfast_inv1(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZFastShape<N1, N2>;
  static_assert((S::NPAIR * 3 * N2) % (2 * S::NTHR) == 0, "tasks in pairs of thread sweeps");
  for (int t = tid; t < S::NPAIR * 3 * N2; t += 2 * nthr) {
    cplx<T> va[N1], vb[N1];
    zfast_inv1_load<T, N1, N2>(c, t, va);
    zfast_inv1_load<T, N1, N2>(c, t + nthr, vb);
    zfast_inv1_finish<T, N1, N2>(c, t, va);
    zfast_inv1_finish<T, N1, N2>(c, t + nthr, vb);
  }
}

// inverse pass 2: thread (g, k1) keeps its positions in registers
template <typename T, int N1, int N2>
NS3D_HD void zfast_inv2(const ZFastCtx<T, N1, N2>& c, int tid, ZFastState<T, N1, N2>& st) {
  using S = ZFastShape<N1, N2>;
  const int k1 = tid % N1;
  const int g = tid / N1;
  st.umax = T(0);
  st.bad = 0;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const cplx<T>* X = c.X + (g * 3 + l) * S::LP;
#pragma unroll
    for (int j = 0; j < N2; ++j) st.z[l][j] = X[j * (N1 + 1) + k1];
    Dft<N2, +1>::run(st.z[l]);
  }
  constexpr bool full = S::P % S::Y == 0;     // every tile has Y columns
  const bool va = full || 2 * g < c.ncol, vb = full || 2 * g + 1 < c.ncol;
  // 0 * s is 0 for finite s and NaN for an infinite or NaN s, so `chk` stays
  // 0 exactly when every point is finite; the maximum skips NaN
  T m = T(0), chk = T(0);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const T sa = xabs(st.z[0][k2].x) + xabs(st.z[0][k2].y) + xabs(st.z[2][k2].x);
    const T sb = xabs(st.z[1][k2].x) + xabs(st.z[1][k2].y) + xabs(st.z[2][k2].y);
    if (va) {
      m = xmax(m, sa);
      chk = chk + T(0) * sa;
    }
    if (vb) {
      m = xmax(m, sb);
      chk = chk + T(0) * sb;
    }
  }
  st.bad = !(chk == T(0)) || !(m <= big_finite<T>());
  st.umax = m;
}

// product line f (0..5) of the pair at register position k2:
// column f % 2, products (00,01), (02,11), (12,22) for f / 2 = 0, 1, 2
template <typename T, int N1, int N2>
NS3D_HD cplx<T> zfast_product(const ZFastState<T, N1, N2>& st, int f, int k2) {
  const int col = f & 1;
  const T u0 = st.z[col][k2].x, u1 = st.z[col][k2].y;
  const T u2 = col ? st.z[2][k2].y : st.z[2][k2].x;
  const int pr = f >> 1;
  if (pr == 0) return cmake(u0 * u0, u0 * u1);
  if (pr == 1) return cmake(u0 * u2, u1 * u1);
  return cmake(u1 * u2, u2 * u2);
}

// forward pass 1 of round r (lines 3r..3r+2): radix N2 over own positions
template <typename T, int N1, int N2>
NS3D_HD void zfast_fwd1(const ZFastCtx<T, N1, N2>& c, int tid, const ZFastState<T, N1, N2>& st,
                        int r) {
  using S = ZFastShape<N1, N2>;
  const int k1 = tid % N1;
  const int g = tid / N1;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    cplx<T> v[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = zfast_product<T, N1, N2>(st, 3 * r + q, k2);
    Dft<N2, -1>::run(v);
    cplx<T>* X = c.X + (g * 3 + q) * S::LP;
#pragma unroll
    for (int k = 0; k < N2; ++k)
      X[k1 * (N2 + 1) + k] = k == 0 ? v[k] : v[k] * c.twf[k * N1 + k1];   // twf[k N1] = 1
  }
}

// forward pass 2: radix N1 in place; tasks (g, q, kappa), kappa < N2
template <typename T, int N1, int N2>
NS3D_HD void zfast_fwd2(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZFastShape<N1, N2>;
  for (int t = tid; t < S::NPAIR * 3 * N2; t += nthr) {
    const int kap = t % N2;
    const int line = t / N2;          // g * 3 + q
    cplx<T>* X = c.X + line * S::LP;
    cplx<T> v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = X[q * (N2 + 1) + kap];
    Dft<N1, -1>::run(v);
#pragma unroll
    for (int k = 0; k < N1; ++k)   // position kap + N2 k; the truncated band is never read
      if (pad_region(N2 * k, N2, S::P, S::H) != PAD_ZERO) X[k * (N2 + 1) + kap] = v[k];
  }
}

// extraction of round r: kz < h of two real lines from each complex line.
// Thread (kl, grp) with kl = tid % KL, grp = tid / KL (6 groups of KL = NTHR/6)
// takes the lines grp + 6 i (all with q = grp % 3) at k = kl + KL j.
template <int N1, int N2>
struct ZExtractShape {
  static constexpr int H = N1 * N2 / 3;
  static constexpr int NG = 6;
  static constexpr int KL = ZFastShape<N1, N2>::NTHR / NG;
  static_assert(ZFastShape<N1, N2>::NTHR == NG * KL && H % KL == 0,
                "extraction: 6 groups of KL threads, KL dividing h");
  static_assert((ZFastShape<N1, N2>::NPAIR * 3) % NG == 0, "extraction: whole line groups");
};

template <typename T, int N1, int N2>
NS3D_HD void zfast_extract(const ZFastCtx<T, N1, N2>& c, int tid, int r) {
  using S = ZFastShape<N1, N2>;
  using E = ZExtractShape<N1, N2>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  cplx<T>* out = a.out + c.bz * a.out_bs + c.by * a.xs + (long long)c.y0 * h;
  const int kl = tid % E::KL, grp = tid / E::KL;
  const int q = grp % 3, f = 3 * r + q;
  const int comp = 2 * (f >> 1);
  cplx<T>* o0 = out + comp * a.out_cs;
  cplx<T>* o1 = out + (comp + 1) * a.out_cs;
  constexpr bool full = S::P % S::Y == 0;
#pragma unroll
  for (int j = 0; j < h / E::KL; ++j) {
    const int k = kl + E::KL * j;
    const int pk = zfast_fpos<N1, N2>(k);
    const int pm = zfast_fpos<N1, N2>(k == 0 ? 0 : S::P - k);
#pragma unroll
    for (int i = 0; i < S::NPAIR * 3 / E::NG; ++i) {
      const int line = grp + E::NG * i;   // g * 3 + q
      const int col = 2 * (line / 3) + (f & 1);
      if (!full && col >= c.ncol) continue;
      const cplx<T>* X = c.X + line * S::LP;
      const cplx<T> zk = X[pk];
      const cplx<T> zm = cconj(X[pm]);
      const cplx<T> s = zk + zm, d = zk - zm;
      o0[col * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
      o1[col * h + k] = cmake(T(0.5) * d.y, T(-0.5) * d.x);
    }
  }
}

// Block maximum of the per-thread maxima (in T: FP64 instructions are slow on
// this part), one atomic per block; a negative entry flags a non-finite value.
// On the GPU warp 0 reduces (lane-strided, then shuffles); the host emulator
// calls it once with lane 0 and reduces serially (max and or are exact in any
// order).
template <typename T, int N1, int N2>
NS3D_HD void zfast_reduce(const ZFastCtx<T, N1, N2>& c, const T* red, int nthr, int lane) {
  const ZArgs<T>& a = *c.a;
  if (!a.ctrl) return;
  T m = T(0);
  int bad = 0;
#if defined(__CUDA_ARCH__)
  for (int i = lane; i < nthr; i += 32) {
    const T r = red[i];
    bad |= r < T(0);
    m = r > m ? r : m;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T o = __shfl_xor_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
#else
  for (int i = 0; i < nthr; ++i) {
    const T r = red[i];
    bad |= r < T(0);
    m = r > m ? r : m;
  }
#endif
  if (lane != 0) return;
  atomic_max_u64(&a.ctrl[c.bz].umax_bits, dbl_bits((double)m));
  if (bad) atomic_or_i32(&a.ctrl[c.bz].status, NS3D_FLAG_NONFINITE);
}
