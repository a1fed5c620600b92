// Fused z pass with three-pass register transforms, for long padded lines
// P = N1 * N2 * N3 (P = 1536 = 24 * 8 * 8 at N = 1024).
//
// Same arithmetic as zfused_block and zfast (Algorithm 2 steps 2-4 along z:
// c2r of the three velocity components with the kz padding, the six products,
// the CFL maximum, r2c truncated to kz < N/2; two real lines per complex
// transform), for one pair of adjacent y columns at a time.  With M = N2 N3:
//
//   inverse 1  task (line, j' < M): radix N1 over positions M j1 + j' read
//              from global memory (zero band pruned at compile time),
//              twiddle w^(j' k1), to slot (j', k1)
//   inverse 2  task (line, k1, j3): radix N2 over slots (N3 j2 + j3, k1),
//              twiddle w^(N1 j3 k2), back to the same slots
//   inverse 3  thread (k1, k2): radix N3 over slots (N3 k2 + j3, k1); the
//              thread keeps the physical values at positions
//              k1 + N1 k2 + N1 N2 k3 of the pair's three lines in registers
//   forward A  thread (a = k1, b = k2): products at its positions, radix N3
//              over k3 (the transposed factorisation), twiddle w^(N1 b f3),
//              to slot (N3 b + f3, a)
//   forward B  task (line, a, f3): radix N2 over slots (N3 b + f3, a),
//              twiddle w^(a (f3 + N3 f2)), back in place
//   forward C  task (line, i = N3 f2 + f3): radix N1 over slots (i, a); the
//              result X[i + M f1] goes to slot (i, f1) where it is kept
//   extraction two real lines from each complex line, kz < h, to global
//
// Slot (i, a) of a line sits at i (N1 + 1) + a: every pass reads and writes
// either consecutive a across lanes or rows of odd stride, so no two lanes of
// a half-warp share a bank.  Blocks are persistent over the (member, x, pair)
// tiles so that the twiddle tables are loaded once per block; the CFL maximum
// is accumulated per thread and reduced when the member changes.  Storage type
// T (global memory), arithmetic type C = LongC<T> (registers, shared memory):
// FP64 data are transformed in double-single arithmetic (ns3d_df64.cuh).
#pragma once

#include "ns3d_blocks.cuh"
#include "ns3d_df64.cuh"

template <> NS3D_HD df64 big_finite<df64>() { return df64(3.4028234663852886e38f); }

// FP32: P = 1536 as 24 x 8 x 8: every phase has a whole number of tasks per
// thread (3 M = N1 N2 with M = N2 N3 = 64), and the zero band kz in [512,
// 1024) is the whole blocks j1 = 8..15 of inverse pass 1
#define NS3D_FOR_ZFAST3(X) X(24, 8, 8)
// FP64 (double-single arithmetic; the compile-time pruning of the padding
// and truncation bands saves arithmetic): P = 192, 384, 1152 (the z pass at
// 384 as 8 x 8 x 6: 10% faster than 16 x 4 x 6 in a standalone timing; at
// 1152 as 12 x 12 x 8: 2 tasks per thread in every phase, and the zero band
// kz in [384, 768) is the whole pass-1 blocks j1 = 4..7)
#define NS3D_FOR_ZFAST3_F64(X) X(16, 4, 3) X(8, 8, 6) X(12, 12, 8)
#define NS3D_FOR_COLFAST3_F64(X) X(16, 4, 3) X(16, 4, 6) X(16, 9, 8)

template <int N1, int N2, int N3>
struct ZFast3Shape {
  static constexpr int P = N1 * N2 * N3;
  static constexpr int H = P / 3;        // N/2 of the default padding P = 3N/2
  static constexpr int M = N2 * N3;
  static constexpr int LR = N1 + 1;      // padded slot row
  static constexpr int LP = M * LR;      // one line
  static constexpr int NTHR = N1 * N2;
  // shared memory (complex elements): T1 [N1][M] inverse pass-1 twiddles,
  // T3 [M][N1] forward pass-B twiddles, w_M^e forward and inverse, 3 lines
  static constexpr int OFF_T3 = P;
  static constexpr int OFF_WM = 2 * P;
  static constexpr int OFF_X = 2 * P + 2 * M;
  static constexpr int SM_ELEMS = OFF_X + 3 * LP;
};

template <typename T, int N1, int N2, int N3>
struct ZFast3State {
  using C = LongC<T>;
  cplx<C> z[3][N3];   // inverse results at positions k1 + N1 k2 + N1 N2 k3
  C umax;             // running max of |u0| + |u1| + |u2| (current member)
  C chk;              // 0 while every point seen is finite
};

template <typename T, int N1, int N2, int N3>
struct ZFast3Ctx {
  using C = LongC<T>;
  const ZArgs<T>* a;
  const cplx<T>* in;   // the pair's first column: [comp][col][kz], col stride h
  cplx<T>* out;
  const cplx<C>* T1;
  const cplx<C>* T3;
  const cplx<C>* wf;   // w_M^e = w_P^(N1 e)
  const cplx<C>* wi;   // conjugate
  cplx<C>* X;
};

// tile t of a launch: member, x row, pair of y columns
template <int N1, int N2, int N3>
NS3D_HD void zfast3_tile(long long t, int* bz, int* by, int* y0) {
  using S = ZFast3Shape<N1, N2, N3>;
  constexpr long long pairs = S::P / 2;
  *y0 = (int)(t % pairs) * 2;
  const long long r = t / pairs;
  *by = (int)(r % S::P);
  *bz = (int)(r / S::P);
}

template <typename T, int N1, int N2, int N3>
NS3D_HD ZFast3Ctx<T, N1, N2, N3> zfast3_ctx(const ZArgs<T>& a, int bz, int by, int y0,
                                            cplx<LongC<T>>* sm) {
  using S = ZFast3Shape<N1, N2, N3>;
  ZFast3Ctx<T, N1, N2, N3> c;
  c.a = &a;
  c.in = a.in + bz * a.in_bs + by * a.xs + (long long)y0 * S::H;
  c.out = a.out + bz * a.out_bs + by * a.xs + (long long)y0 * S::H;
  c.T1 = sm;
  c.T3 = sm + S::OFF_T3;
  c.wf = sm + S::OFF_WM;
  c.wi = sm + S::OFF_WM + S::M;
  c.X = sm + S::OFF_X;
  return c;
}

template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_twiddles(const ZArgs<T>& a, cplx<LongC<T>>* sm, int tid, int nthr) {
  using S = ZFast3Shape<N1, N2, N3>;
  using C = LongC<T>;
  for (int e = tid; e < S::P; e += nthr) {
    const int k1 = e / S::M, jp = e % S::M;       // T1[k1][j'] = conj w^(j' k1)
    const cplx<T> w1 = a.tw[jp * k1];
    sm[e] = ccvt<C>(cmake(w1.x, -w1.y));
    const int i = e / N1, aa = e % N1;            // T3[i][a] = w^(a i)
    sm[S::OFF_T3 + e] = ccvt<C>(a.tw[aa * i]);
  }
  for (int e = tid; e < S::M; e += nthr) {
    const cplx<T> w = a.tw[N1 * e];
    sm[S::OFF_WM + e] = ccvt<C>(w);
    sm[S::OFF_WM + S::M + e] = ccvt<C>(cmake(w.x, -w.y));
  }
}

// inverse pass 1: tasks (line l, j'), j' fastest (consecutive kz)
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_inv1(const ZFast3Ctx<T, N1, N2, N3>& c, int tid, int nthr) {
  using S = ZFast3Shape<N1, N2, N3>;
  using C = LongC<T>;
  constexpr int h = S::H, M = S::M;
  const ZArgs<T>& a = *c.a;
  for (int t = tid; t < 3 * M; t += nthr) {
    const int jp = t % M, l = t / M;
    // lines: u0 + i u1 of column 0, of column 1, u2(0) + i u2(1)
    const int ca = l == 1 ? 1 : 0, cb = l == 0 ? 0 : 1;
    const cplx<T>* ia = c.in + (l == 2 ? 2 : 0) * a.in_cs + ca * h;
    const cplx<T>* ib = c.in + (l == 2 ? 2 : 1) * a.in_cs + cb * h;
    cplx<C> v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int p = M * j1 + jp;
      const int reg = pad_region(M * j1, M, S::P, S::H);
      if (reg == PAD_ZERO) {
        v[j1] = czero<C>();
      } else if (reg == PAD_LOW) {               // u_a[p] + i u_b[p]
        cplx<C> x = ccvt<C>(ia[p]), y = ccvt<C>(ib[p]);
        if (j1 == 0 && jp == 0) {                // a real line has a real mean
          x.y = C(0);
          y.y = C(0);
        }
        v[j1] = cmake(x.x - y.y, x.y + y.x);
      } else if (reg == PAD_HIGH) {              // conj(u_a[P-p]) + i conj(u_b[P-p])
        const cplx<C> x = ccvt<C>(ia[S::P - p]), y = ccvt<C>(ib[S::P - p]);
        v[j1] = cmake(x.x + y.y, -x.y + y.x);
      } else {
        v[j1] = ccvt<C>(pack2(ia, ib, S::P, S::H, p, 0, 0, 1));
      }
    }
    Dft<N1, +1>::run(v);
    cplx<C>* D = c.X + l * S::LP + jp * S::LR;
    const cplx<C>* tw = c.T1 + jp;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) D[k1] = k1 == 0 ? v[k1] : v[k1] * tw[k1 * M];
  }
}

// inverse pass 2: tasks (line, k1, j3), k1 fastest
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_inv2(const ZFast3Ctx<T, N1, N2, N3>& c, int tid, int nthr) {
  using S = ZFast3Shape<N1, N2, N3>;
  for (int t = tid; t < 3 * N1 * N3; t += nthr) {
    const int k1 = t % N1, j3 = (t / N1) % N3, l = t / (N1 * N3);
    cplx<LongC<T>>* D = c.X + l * S::LP + j3 * S::LR + k1;
    cplx<LongC<T>> v[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) v[j2] = D[j2 * N3 * S::LR];
    Dft<N2, +1>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) D[k2 * N3 * S::LR] = k2 == 0 ? v[k2] : v[k2] * c.wi[j3 * k2];
  }
}

// inverse pass 3: thread (k1, k2) keeps its positions; CFL maximum
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_inv3(const ZFast3Ctx<T, N1, N2, N3>& c, int tid,
                         ZFast3State<T, N1, N2, N3>& st) {
  using S = ZFast3Shape<N1, N2, N3>;
  using C = LongC<T>;
  const int k1 = tid % N1, k2 = tid / N1;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const cplx<C>* D = c.X + l * S::LP + k2 * N3 * S::LR + k1;
#pragma unroll
    for (int j3 = 0; j3 < N3; ++j3) st.z[l][j3] = D[j3 * S::LR];
    Dft<N3, +1>::run(st.z[l]);
  }
  // 0 * s is NaN exactly when s is not finite
#pragma unroll
  for (int k3 = 0; k3 < N3; ++k3) {
    const C sa = xabs(st.z[0][k3].x) + xabs(st.z[0][k3].y) + xabs(st.z[2][k3].x);
    const C sb = xabs(st.z[1][k3].x) + xabs(st.z[1][k3].y) + xabs(st.z[2][k3].y);
    st.umax = xmax(st.umax, xmax(sa, sb));
    st.chk = st.chk + C(0) * sa + C(0) * sb;
  }
}

// product line f (0..5) at register position k3: column f % 2, products
// (00, 01), (02, 11), (12, 22) for f / 2 = 0, 1, 2
template <typename T, int N1, int N2, int N3>
NS3D_HD cplx<LongC<T>> zfast3_product(const ZFast3State<T, N1, N2, N3>& st, int f, int k3) {
  using C = LongC<T>;
  const int col = f & 1;
  const C u0 = st.z[col][k3].x, u1 = st.z[col][k3].y;
  const C u2 = col ? st.z[2][k3].y : st.z[2][k3].x;
  const int pr = f >> 1;
  if (pr == 0) return cmake(u0 * u0, u0 * u1);
  if (pr == 1) return cmake(u0 * u2, u1 * u1);
  return cmake(u1 * u2, u2 * u2);
}

// forward pass A of round r (lines 3r .. 3r + 2)
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_fwdA(const ZFast3Ctx<T, N1, N2, N3>& c, int tid,
                         const ZFast3State<T, N1, N2, N3>& st, int r) {
  using S = ZFast3Shape<N1, N2, N3>;
  const int a = tid % N1, b = tid / N1;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    cplx<LongC<T>> v[N3];
#pragma unroll
    for (int k3 = 0; k3 < N3; ++k3) v[k3] = zfast3_product<T, N1, N2, N3>(st, 3 * r + q, k3);
    Dft<N3, -1>::run(v);
    cplx<LongC<T>>* D = c.X + q * S::LP + N3 * b * S::LR + a;
#pragma unroll
    for (int f3 = 0; f3 < N3; ++f3) D[f3 * S::LR] = f3 == 0 ? v[f3] : v[f3] * c.wf[b * f3];
  }
}

// forward pass B: tasks (line, a, f3), a fastest
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_fwdB(const ZFast3Ctx<T, N1, N2, N3>& c, int tid, int nthr) {
  using S = ZFast3Shape<N1, N2, N3>;
  for (int t = tid; t < 3 * N1 * N3; t += nthr) {
    const int a = t % N1, f3 = (t / N1) % N3, q = t / (N1 * N3);
    cplx<LongC<T>>* D = c.X + q * S::LP + f3 * S::LR + a;
    cplx<LongC<T>> v[N2];
#pragma unroll
    for (int b = 0; b < N2; ++b) v[b] = D[b * N3 * S::LR];
    Dft<N2, -1>::run(v);
    const cplx<LongC<T>>* tw = c.T3 + f3 * N1 + a;      // T3[f3 + N3 f2][a]
#pragma unroll
    for (int f2 = 0; f2 < N2; ++f2) D[f2 * N3 * S::LR] = v[f2] * tw[f2 * N3 * N1];
  }
}

// forward pass C: tasks (line, i), i fastest; the truncated band is not kept
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_fwdC(const ZFast3Ctx<T, N1, N2, N3>& c, int tid, int nthr) {
  using S = ZFast3Shape<N1, N2, N3>;
  for (int t = tid; t < 3 * S::M; t += nthr) {
    const int i = t % S::M, q = t / S::M;
    cplx<LongC<T>>* D = c.X + q * S::LP + i * S::LR;
    cplx<LongC<T>> v[N1];
#pragma unroll
    for (int aa = 0; aa < N1; ++aa) v[aa] = D[aa];
    Dft<N1, -1>::run(v);
#pragma unroll
    for (int f1 = 0; f1 < N1; ++f1)   // natural position i + M f1
      if (pad_region(S::M * f1, S::M, S::P, S::H) != PAD_ZERO) D[f1] = v[f1];
  }
}

// slot of natural forward position k
template <int N1, int N2, int N3>
NS3D_HD int zfast3_fpos(int k) {
  using S = ZFast3Shape<N1, N2, N3>;
  return (k % S::M) * S::LR + k / S::M;
}

// extraction of round r: kz < h of two real lines from each complex line
template <typename T, int N1, int N2, int N3>
NS3D_HD void zfast3_extract(const ZFast3Ctx<T, N1, N2, N3>& c, int tid, int nthr, int r) {
  using S = ZFast3Shape<N1, N2, N3>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  for (int t = tid; t < 3 * h; t += nthr) {
    const int k = t % h, q = t / h;
    const int f = 3 * r + q;
    const int col = f & 1, comp = 2 * (f >> 1);
    using C = LongC<T>;
    const cplx<C>* X = c.X + q * S::LP;
    const cplx<C> zk = X[zfast3_fpos<N1, N2, N3>(k)];
    const cplx<C> zm = cconj(X[zfast3_fpos<N1, N2, N3>(k == 0 ? 0 : S::P - k)]);
    const cplx<C> s = zk + zm, d = zk - zm;
    c.out[comp * a.out_cs + col * h + k] = ccvt<T>(cmake(C(0.5) * s.x, C(0.5) * s.y));
    c.out[(comp + 1) * a.out_cs + col * h + k] = ccvt<T>(cmake(C(0.5) * d.y, C(-0.5) * d.x));
  }
}

// CFL maximum of member bz from the per-thread values in red (negative: a
// non-finite value was seen).  GPU: warp 0 reduces; host emulation: lane 0,
// serially (max and or are exact in any order).
template <typename T>
NS3D_HD void zfast3_flush(const ZArgs<T>& a, int bz, const T* red, int nthr, int lane) {
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
  atomic_max_u64(&a.ctrl[bz].umax_bits, dbl_bits((double)m));
  if (bad) atomic_or_i32(&a.ctrl[bz].status, NS3D_FLAG_NONFINITE);
}

template <typename T, int N1, int N2, int N3>
NS3D_HD T zfast3_red_value(const ZFast3State<T, N1, N2, N3>& st) {
  using C = LongC<T>;
  return (!(st.chk == C(0)) || !(st.umax <= big_finite<C>())) ? T(-1) : (T)st.umax;
}
