// Block bodies of the solver's kernels (one CUDA block each).
//
// Every function here takes the block index, the thread index/count, a
// shared-memory pointer and a barrier functor, so the same code runs as a
// CUDA block (kernels_*.cu) and, block by block with one emulated thread, on
// the CPU (hostcheck.cpp) where the tests compare it with the oracle.
//
// Data layout in device memory (per ensemble level: B members of size N, padded
// size P, h = N/2; all complex, interleaved re/im):
//   state   U  [B][3][kx N][ky N][kz h]    retained modes; kz = N/2 is dropped,
//                                         rows kx = h and ky = h stay zero
//   A  (inverse x done)   [B][3][x P][ky N][kz h]
//   Bq (inverse x,y done) [B][3][x P][y P][kz h]
//   Cq (products, fwd z)  [B][6][x P][y P][kz h]
//   Dq (fwd z,y)          [B][6][x P][ky N][kz h]
//   Bh (fwd z,y,x)        [B][6][kx N][ky N][kz h]
// The product components are ordered B00 B01 B02 B11 B12 B22.
#pragma once

#include "ns3d_fft.cuh"

NS3D_HD int imin(int a, int b) { return a < b ? a : b; }
// largest finite value of T: v <= big_finite<T>() is false for NaN and +-inf
template <typename T> NS3D_HD T big_finite();
template <> NS3D_HD float big_finite<float>() { return 3.4028234663852886e38f; }
template <> NS3D_HD double big_finite<double>() { return 1.7976931348623157e308; }
NS3D_HD float xabs(float a) { return fabsf(a); }
NS3D_HD double xabs(double a) { return fabs(a); }
NS3D_HD float xpow(float a, float b) { return powf(a, b); }
// maximum that ignores a NaN operand
NS3D_HD float xmax(float a, float b) { return fmaxf(a, b); }
NS3D_HD double xmax(double a, double b) { return fmax(a, b); }
NS3D_HD double xpow(double a, double b) { return pow(a, b); }

// Per-member control word kept in device memory.
struct Ns3dCtrl {
  double t;                      // time reached
  double dt;                     // time step of the step in progress (set at stage 1)
  double t_end;                  // stop time (<= 0: none); a member at t_end stays put
  unsigned long long umax_bits;  // max_x sum_i |u_i| of the stage-1 field (double bits)
  int status;                    // sticky NS3D_FLAG_* bits
  int nsteps;                    // completed steps
  float dtf;                     // dt rounded to float (read by the FP32 stage kernels)
  int pad_;
};

#define NS3D_FLAG_NONFINITE 1
#define NS3D_FLAG_UNSTABLE 2
#define NS3D_FLAG_TIMEOUT 4   // a staged copy did not arrive within its time limit

NS3D_HD void atomic_max_u64(unsigned long long* p, unsigned long long v) {
#if defined(__CUDA_ARCH__)
  atomicMax(p, v);
#else
  if (*p < v) *p = v;
#endif
}

NS3D_HD void atomic_or_i32(int* p, int v) {
#if defined(__CUDA_ARCH__)
  atomicOr(p, v);
#else
  *p |= v;
#endif
}

NS3D_HD unsigned long long dbl_bits(double d) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(d);
#else
  union { double d; unsigned long long u; } c;
  c.d = d;
  return c.u;
#endif
}

NS3D_HD double bits_dbl(unsigned long long u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  union { double d; unsigned long long u; } c;
  c.u = u;
  return c.d;
#endif
}

// =====================================================================
// Column pass: 1D transforms along one axis of a strided array
// (Algorithm 3 steps 1-2 for the inverse with padding; the forward transform
// with truncation is Algorithm 3 run in reverse, "remove the upper third").
// =====================================================================
template <typename T>
struct ColArgs {
  const cplx<T>* in;
  cplx<T>* out;
  const cplx<T>* tw;     // exp(-2 pi i e / n), e < n
  FftPlanDev pl;
  int h;                 // N/2
  int nrow_in, nrow_out; // rows of the input / output arrays along the axis
  int pad_in;            // input has N rows, spread over the n positions (zero pad)
  int trunc_out;         // output keeps N rows of the n positions
  int ncols;             // columns per (batch, outer) slice
  int W, ldw;            // columns per block, padded shared row length
  long long in_bs, in_os, in_cs, in_rs;    // batch / outer / column / row strides
  long long out_bs, out_os, out_cs, out_rs;
  T scale;
};

template <typename T>
struct ColLoad {
  const cplx<T>* in;
  long long cs, rs;
  int n, h, nrow, pad;
  NS3D_HD cplx<T> operator()(int col, int p) const {
    const int row = pad ? pad_row_of(p, n, h, nrow) : p;
    if (row < 0) return czero<T>();
    return in[col * cs + row * rs];
  }
};

template <typename T>
struct ColStore {
  cplx<T>* out;
  long long cs, rs;
  int n, h, nrow, trunc;
  T scale;
  NS3D_HD void operator()(int col, int p, cplx<T> v) const {
    const int row = trunc ? pad_row_of(p, n, h, nrow) : p;
    if (row >= 0) out[col * cs + row * rs] = scale * v;
  }
};

template <typename T, int SIGN, bool CF_FIRST, bool CF_LAST, class Sync>
NS3D_HD void colfft_block(const ColArgs<T>& a, int bx, int by, int bz, int tid, int nthr,
                          cplx<T>* sm, const Sync& sync) {
  const int c0 = bx * a.W;
  const int ncol = imin(a.W, a.ncols - c0);
  if (ncol <= 0) return;
  const cplx<T>* in = a.in + bz * a.in_bs + by * a.in_os + c0 * a.in_cs;
  cplx<T>* out = a.out + bz * a.out_bs + by * a.out_os + c0 * a.out_cs;
  const int n = a.pl.n;
  ColLoad<T> ld{in, a.in_cs, a.in_rs, n, a.h, a.nrow_in, a.pad_in};
  ColStore<T> st{out, a.out_cs, a.out_rs, n, a.h, a.nrow_out, a.trunc_out, a.scale};
  fft_tile<T, SIGN, CF_FIRST, CF_LAST>(a.pl, ncol, tid, nthr, a.tw, ld, st, sm, sm + n * a.ldw,
                                       a.ldw, sync);
  if (a.trunc_out) {
    // the Nyquist row N/2 receives no position: keep it zero
    for (int col = tid; col < ncol; col += nthr) out[col * a.out_cs + a.h * a.out_rs] = czero<T>();
  }
}

// =====================================================================
// Fused z pass (Algorithm 2 steps 2-4 along the last axis): complex-to-real
// inverse of the three velocity components with the kz padding, the six
// products B_jl = u_j u_l on the padded grid, the CFL maximum, and the
// real-to-complex forward transform truncated to kz < N/2.  Two real lines
// share one complex transform (z = a + i b; A_k = (Z_k + conj Z_{n-k})/2,
// B_k = (Z_k - conj Z_{n-k})/(2i)).  Nothing physical is written to memory.
// =====================================================================
template <typename T>
struct ZArgs {
  const cplx<T>* in;   // Bq
  cplx<T>* out;        // Cq
  const cplx<T>* tw;   // length P
  FftPlanDev pl;
  int P, h, W, ldw;
  long long in_bs, in_cs;    // member / component strides of Bq
  long long out_bs, out_cs;  // member / component strides of Cq
  long long xs;              // x stride (h * P) of both
  Ns3dCtrl* ctrl;            // per member (null: no CFL reduction)
};

// u_a + i u_b packed spectrum at position p of a length-P line, from the
// stored half spectra of lines ca and cb (line c, wavenumber q at c*h + q)
template <typename T>
NS3D_HD cplx<T> pack2(const cplx<T>* ia, const cplx<T>* ib, int P, int h, int p, int ca, int cb,
                      int ncol) {
  cplx<T> a = czero<T>(), b = czero<T>();
  if (p < h) {
    if (ca < ncol) a = ia[ca * h + p];
    if (cb < ncol) b = ib[cb * h + p];
    if (p == 0) {
      a.y = T(0);   // a real line has a real mean: keep the Hermitian part
      b.y = T(0);
    }
  } else if (p > P - h) {
    const int q = P - p;
    if (ca < ncol) a = cconj(ia[ca * h + q]);
    if (cb < ncol) b = cconj(ib[cb * h + q]);
  } else {
    return czero<T>();
  }
  return cmake(a.x - b.y, a.y + b.x);
}

template <typename T>
struct ZLoadInv {
  const cplx<T>* ia;
  const cplx<T>* ib;
  int P, h, ncol, pair_off;  // pair_off = 0: (u0,u1) same column; else u2 columns (m, m+off)
  NS3D_HD cplx<T> operator()(int col, int p) const {
    if (pair_off == 0) return pack2(ia, ib, P, h, p, col, col, ncol);
    return pack2(ia, ib, P, h, p, col, col + pair_off, ncol);
  }
};

// (line a + i line b) of the same column; off != 0 makes b zero
template <typename T>
struct ZLoadInvCols {
  const cplx<T>* ia;
  const cplx<T>* ib;
  int P, h, ncol, off;
  NS3D_HD cplx<T> operator()(int col, int p) const {
    return pack2(ia, ib, P, h, p, col, col + off, ncol);
  }
};

template <typename T>
struct ZPhys {  // physical velocity at (position p, column col) from the inverse results
  const cplx<T>* U01;
  const cplx<T>* U2;
  int ldw, half;
  NS3D_HD void get(int col, int p, T& u0, T& u1, T& u2) const {
    const cplx<T> z = U01[p * ldw + col];
    u0 = z.x;
    u1 = z.y;
    u2 = (col < half) ? U2[p * ldw + col].x : U2[p * ldw + col - half].y;
  }
};

template <typename T>
struct ZLoadProd {
  ZPhys<T> ph;
  int pair;
  NS3D_HD cplx<T> operator()(int col, int p) const {
    T u0, u1, u2;
    ph.get(col, p, u0, u1, u2);
    if (pair == 0) return cmake(u0 * u0, u0 * u1);
    if (pair == 1) return cmake(u0 * u2, u1 * u1);
    return cmake(u1 * u2, u2 * u2);
  }
};

// CFL maximum of one tile: max over its points of sum_i |u_i| (`get` gives the
// velocity at (column, position)) into the member's control word, or the
// non-finite flag.
template <typename T, class Get, class Sync>
NS3D_HD void z_umax_reduce(Ns3dCtrl* ctrl, int P, int ncol, int tid, int nthr, double* red,
                           const Get& ph, const Sync& sync) {
  T m = T(0);
  int bad = 0;
  for (int w = tid; w < P * ncol; w += nthr) {
    const int col = w % ncol, p = w / ncol;
    T u0, u1, u2;
    ph.get(col, p, u0, u1, u2);
    const T s = xabs(u0) + xabs(u1) + xabs(u2);
    if (!(s <= big_finite<T>())) bad = 1;
    else m = s > m ? s : m;
  }
  T* tred = reinterpret_cast<T*>(red);
  tred[tid] = bad ? T(-1) : m;
  sync();
  if (tid == 0) {
    T mm = T(0);
    int anybad = 0;
    for (int i = 0; i < nthr; ++i) {
      const T r = tred[i];
      anybad |= r < T(0);
      mm = r > mm ? r : mm;
    }
    atomic_max_u64(&ctrl->umax_bits, dbl_bits((double)mm));
    if (anybad) atomic_or_i32(&ctrl->status, NS3D_FLAG_NONFINITE);
  }
}

template <typename T, class Sync>
NS3D_HD void zfused_block(const ZArgs<T>& a, int bx, int by, int bz, int tid, int nthr,
                          cplx<T>* sm, double* red, const Sync& sync) {
  const int P = a.P, h = a.h, W = a.W, ldw = a.ldw;
  const int y0 = bx * W;
  const int ncol = imin(W, P - y0);
  const int half = W / 2;
  cplx<T>* U01 = sm;
  cplx<T>* U2 = sm + P * ldw;
  cplx<T>* A = sm + 2 * P * ldw;
  cplx<T>* B = sm + 3 * P * ldw;
  const cplx<T>* in = a.in + bz * a.in_bs + by * a.xs + (long long)y0 * h;
  SmemIO<T> u01{U01, ldw}, u2s{U2, ldw};

  // inverse: (u0 + i u1) per column, and u2 of columns (m, m + W/2) per pair;
  // lines are contiguous along kz, so the first pass maps positions fastest
  ZLoadInv<T> l01{in, in + a.in_cs, P, h, ncol, 0};
  fft_tile<T, +1, false, true>(a.pl, ncol, tid, nthr, a.tw, l01, u01, A, B, ldw, sync);
  sync();
  ZLoadInv<T> l22{in + 2 * a.in_cs, in + 2 * a.in_cs, P, h, ncol, half};
  fft_tile<T, +1, false, true>(a.pl, half, tid, nthr, a.tw, l22, u2s, A, B, ldw, sync);
  sync();

  ZPhys<T> ph{U01, U2, ldw, half};
  if (a.ctrl) z_umax_reduce<T>(a.ctrl + bz, P, ncol, tid, nthr, red, ph, sync);

  // forward: three packed pairs of products, each truncated to kz < h
  cplx<T>* out = a.out + bz * a.out_bs + by * a.xs + (long long)y0 * h;
  for (int pair = 0; pair < 3; ++pair) {
    ZLoadProd<T> lp{ph, pair};
    cplx<T>* E = fft_free_buffer(a.pl.npass, A, B);
    SmemIO<T> e{E, ldw};
    fft_tile<T, -1, true, true>(a.pl, ncol, tid, nthr, a.tw, lp, e, A, B, ldw, sync);
    sync();
    cplx<T>* oa = out + (2 * pair) * a.out_cs;
    cplx<T>* ob = out + (2 * pair + 1) * a.out_cs;
    for (int w = tid; w < h * ncol; w += nthr) {
      const int k = w % h, col = w / h;
      const cplx<T> zk = E[k * ldw + col];
      const cplx<T> zm = cconj(E[((P - k) % P) * ldw + col]);
      const cplx<T> s = zk + zm;
      const cplx<T> d = zk - zm;
      oa[col * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
      ob[col * h + k] = cmake(T(0.5) * d.y, T(-0.5) * d.x);   // d / (2i)
    }
    sync();
  }
}

// =====================================================================
// The advective and rotational forms of the nonlinear term.  For a
// divergence-free field with 3/2 padding both equal the divergence form after
// the Leray projection, up to rounding:
//   form 1  b = -F[(u . grad) u],   (u . grad) u_j = sum_l u_l d_l u_j
//   form 2  b =  F[u x omega],      omega = curl u
// (u x omega = -(u . grad) u + grad |u|^2 / 2, and a gradient projects out).
// The fields taken to the padded grid: form 1 u_j and d_l u_j (field
// 3 + 3 l + j), twelve; form 2 u_j and omega_j (field 3 + j), six.  The z pass
// forms the three products in shared memory and returns them by two forward
// transforms: (p0 + i p1) and p2.
// =====================================================================

NS3D_HDC int form_fields(int form) { return form == 1 ? 12 : (form == 2 ? 6 : 3); }

// the spectral fields of one mode i of the compact [3][N][N][h] layout, into
// F [nf][N][N][h]: u_hat itself, then i kappa_l u_hat_j (form 1) or
// i kappa x u_hat (form 2)
template <typename T>
NS3D_HD void form_prep_point(const cplx<T>* u, cplx<T>* F, int N, T kscale, int form, long long i) {
  const int h = N / 2;
  const long long plane = (long long)N * N * h;
  const int kz = (int)(i % h);
  const int ky = (int)((i / h) % N), kx = (int)(i / ((long long)h * N));
  const T k0 = kscale * T(kx < h ? kx : kx - N), k1 = kscale * T(ky < h ? ky : ky - N),
          k2 = kscale * T(kz);
  const cplx<T> v0 = u[i], v1 = u[plane + i], v2 = u[2 * plane + i];
  F[i] = v0;
  F[plane + i] = v1;
  F[2 * plane + i] = v2;
  if (form == 1) {
    const T kl[3] = {k0, k1, k2};
    const cplx<T> vj[3] = {v0, v1, v2};
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int j = 0; j < 3; ++j)   // i a (x + iy) = -a y + i a x
        F[(3 + 3 * l + j) * plane + i] = cmake(-kl[l] * vj[j].y, kl[l] * vj[j].x);
  } else {
    const cplx<T> c0 = k1 * v2 - k2 * v1, c1 = k2 * v0 - k0 * v2, c2 = k0 * v1 - k1 * v0;
    F[3 * plane + i] = cmake(-c0.y, c0.x);
    F[4 * plane + i] = cmake(-c1.y, c1.x);
    F[5 * plane + i] = cmake(-c2.y, c2.x);
  }
}

// Inverse transforms of the z pass, in order: the fields (a, b) packed as
// a + i b, one pair per transform (form 1: six, form 2: three).
NS3D_HD void form_pair(int form, int step, int* a, int* b) {
  // form 1: (u0,u1) (u2,d0u0) (d1u0,d2u0) (d0u1,d1u1) (d2u1,d0u2) (d1u2,d2u2)
  const int f1[12] = {0, 1, 2, 3, 6, 9, 4, 7, 10, 5, 8, 11};
  // form 2: (u0,u1) (u2,w0) (w1,w2)
  const int f2[6] = {0, 1, 2, 3, 4, 5};
  *a = form == 1 ? f1[2 * step] : f2[2 * step];
  *b = form == 1 ? f1[2 * step + 1] : f2[2 * step + 1];
}

// Last pass of each inverse transform: the value v = a + i b at (column,
// position) goes into the product buffers.  U01 = u0 + i u1 throughout;
// X = u2 + i (form 1: N2, form 2: w0); form 1's Y = N0 + i N1, with
// N_j = sum_l u_l d_l u_j.  After the last step the products are
// form 1: Y = N0 + i N1, X = N2; form 2: U01 = p0 + i p1, X = p2 (p = u x w).
template <typename T>
struct ZFormStore {
  cplx<T>* U01;
  cplx<T>* X;
  cplx<T>* Y;
  int ldw, form, step;
  NS3D_HD void operator()(int col, int f, cplx<T> v) const {
    const int o = f * ldw + col;
    if (step == 0) {
      U01[o] = v;
      return;
    }
    const cplx<T> uu = U01[o];
    const T u0 = uu.x, u1 = uu.y;
    if (form == 2) {
      if (step == 1) {
        X[o] = v;
        return;
      }
      const cplx<T> xw = X[o];
      const T u2 = xw.x, w0 = xw.y, w1 = v.x, w2 = v.y;
      U01[o] = cmake(u1 * w2 - u2 * w1, u2 * w0 - u0 * w2);
      X[o] = cmake(u0 * w1 - u1 * w0, T(0));
      return;
    }
    if (step == 1) {                        // (u2, d0 u0)
      X[o] = cmake(v.x, T(0));
      Y[o] = cmake(u0 * v.y, T(0));
      return;
    }
    const cplx<T> xw = X[o];
    const T u2 = xw.x;
    cplx<T> y = Y[o];
    if (step == 2) {                        // (d1 u0, d2 u0)
      y.x += u1 * v.x + u2 * v.y;
      Y[o] = y;
    } else if (step == 3) {                 // (d0 u1, d1 u1)
      y.y = u0 * v.x + u1 * v.y;
      Y[o] = y;
    } else if (step == 4) {                 // (d2 u1, d0 u2)
      y.y += u2 * v.x;
      Y[o] = y;
      X[o] = cmake(u2, u0 * v.y);
    } else {                                // (d1 u2, d2 u2): N2 done, u2 no longer needed
      X[o] = cmake(xw.y + u1 * v.x + u2 * v.y, T(0));
    }
  }
};

template <typename T>
struct ZFormPhys {  // velocity after the second inverse transform
  const cplx<T>* U01;
  const cplx<T>* X;
  int ldw;
  NS3D_HD void get(int col, int p, T& u0, T& u1, T& u2) const {
    const cplx<T> z = U01[p * ldw + col];
    u0 = z.x;
    u1 = z.y;
    u2 = X[p * ldw + col].x;
  }
};

// Shared elements of a zform tile: the product buffers (form 1: U01, X, Y;
// form 2: U01, X) and the two transform buffers, P (W + 1) elements each.
NS3D_HDC int zform_buffers(int form) { return form == 1 ? 5 : 4; }

// z pass of forms 1 and 2 for one tile of W y columns at (member bz, x = by):
// in [m][nf][P][P][h] (the inverse x and y of the form's fields), out
// [m][3][P][P][h] the truncated half spectra of the three products.
template <typename T, class Sync>
NS3D_HD void zform_block(const ZArgs<T>& a, int form, int bx, int by, int bz, int tid, int nthr,
                         cplx<T>* sm, double* red, const Sync& sync) {
  const int P = a.P, h = a.h, W = a.W, ldw = a.ldw;
  const int y0 = bx * W;
  const int ncol = imin(W, P - y0);
  const int nprod = form == 1 ? 3 : 2;
  cplx<T>* U01 = sm;
  cplx<T>* X = sm + P * ldw;
  cplx<T>* Y = sm + 2 * P * ldw;            // form 1 only
  cplx<T>* A = sm + nprod * P * ldw;
  cplx<T>* B = A + P * ldw;
  const cplx<T>* in = a.in + bz * a.in_bs + by * a.xs + (long long)y0 * h;
  const int nsteps = form == 1 ? 6 : 3;
  for (int st = 0; st < nsteps; ++st) {
    int fa, fb;
    form_pair(form, st, &fa, &fb);
    ZLoadInvCols<T> ld{in + fa * a.in_cs, in + fb * a.in_cs, P, h, ncol, 0};
    ZFormStore<T> sto{U01, X, Y, ldw, form, st};
    fft_tile<T, +1, false, true>(a.pl, ncol, tid, nthr, a.tw, ld, sto, A, B, ldw, sync);
    sync();
    if (st == 1 && a.ctrl) {
      ZFormPhys<T> ph{U01, X, ldw};
      z_umax_reduce<T>(a.ctrl + bz, P, ncol, tid, nthr, red, ph, sync);
      sync();
    }
  }
  // forward: (p0 + i p1) untangled into two half spectra, then p2 alone
  cplx<T>* out = a.out + bz * a.out_bs + by * a.xs + (long long)y0 * h;
  for (int pair = 0; pair < 2; ++pair) {
    SmemIO<T> src{pair == 0 ? (form == 1 ? Y : U01) : X, ldw};
    cplx<T>* E = fft_free_buffer(a.pl.npass, A, B);
    SmemIO<T> e{E, ldw};
    fft_tile<T, -1, true, true>(a.pl, ncol, tid, nthr, a.tw, src, e, A, B, ldw, sync);
    sync();
    cplx<T>* oa = out + (2 * pair) * a.out_cs;
    cplx<T>* ob = out + (2 * pair + 1) * a.out_cs;
    for (int w = tid; w < h * ncol; w += nthr) {
      const int k = w % h, col = w / h;
      const cplx<T> zk = E[k * ldw + col];
      const cplx<T> zm = cconj(E[((P - k) % P) * ldw + col]);
      const cplx<T> s = zk + zm;
      oa[col * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
      if (pair == 0) {
        const cplx<T> d = zk - zm;
        ob[col * h + k] = cmake(T(0.5) * d.y, T(-0.5) * d.x);   // d / (2i)
      }
    }
    sync();
  }
}

// =====================================================================
// Spectral step (section 2.3 and eq. RK3): b = -i kappa . B_hat / P^3,
// Leray projection, dissipation lambda_k u_k, and the SSP-RK3 stage combine.
// =====================================================================
struct SpecParams {
  double kscale;      // 2 pi / L
  double nu, epsN, s, mN2, qexp;
  int kthr;           // |k|^2 <= kthr: no hyper-viscosity
  int q_form;
  double inv_P3;
  double cfl, dx, dt_fixed, lam_max;
};


NS3D_HD double member_dt(const Ns3dCtrl& c, const SpecParams& sp) {
  double dt;
  const double umax = bits_dbl(c.umax_bits);
  if (sp.dt_fixed > 0) dt = sp.dt_fixed;
  else if (umax > 0) dt = sp.cfl * sp.dx / umax;
  else dt = (c.t_end > 0) ? c.t_end - c.t : 0.0;
  if (c.t_end > 0) {
    const double rem = c.t_end - c.t;
    if (dt > rem) dt = rem;
    if (dt < 0) dt = 0;
  }
  return dt;
}

// Start of a step for member m (one thread per member, before the stage-1
// spectral kernel): the step's dt from the CFL maximum of the stage-1 field,
// and the stability check lambda_max dt <= 2.5.
NS3D_HD void step_dt_member(Ns3dCtrl& c, const SpecParams& sp) {
  const double dt = member_dt(c, sp);
  c.dt = dt;
  c.dtf = (float)dt;
  if (dt * sp.lam_max > 2.5) c.status |= NS3D_FLAG_UNSTABLE;
}

// The spectral parameters in the arithmetic type, converted once per thread.
template <typename T>
struct SpecT {
  T kscale, nu, epsN, s, mN2, qexp, inv_P3;
  int kthr, q_form;
};

template <typename T>
NS3D_HD SpecT<T> spec_t(const SpecParams& sp) {
  SpecT<T> r;
  r.kscale = (T)sp.kscale;
  r.nu = (T)sp.nu;
  r.epsN = (T)sp.epsN;
  r.s = (T)sp.s;
  r.mN2 = (T)sp.mN2;
  r.qexp = (T)sp.qexp;
  r.inv_P3 = (T)sp.inv_P3;
  r.kthr = sp.kthr;
  r.q_form = sp.q_form;
  return r;
}

template <typename T>
NS3D_HD T lambda_k(int k2, const SpecT<T>& sp) {
  const T kap2 = sp.kscale * sp.kscale * T(k2);
  T lam = sp.nu * kap2;
  if (k2 > sp.kthr) {
    T q = T(1);
    if (sp.q_form == 0) q = T(1) - xpow(sp.mN2 / T(k2), sp.qexp);
    lam += sp.epsN * xpow(kap2, sp.s) * q;
  }
  return lam;
}

template <typename T>
struct SpecArgs {
  const cplx<T>* bh;   // Bh
  const cplx<T>* u0;   // U at t_n
  const cplx<T>* us;   // stage state (stages 2, 3)
  cplx<T>* out;        // next stage / next state / R (stage 0)
  int N, h, nmem;
  int stage;           // 0: out = R; 1, 2, 3: RK3 stages (dt from ctrl)
  long long m6, m3;    // member strides of Bh and of U
  SpecT<T> sp;         // parameters in the arithmetic type
  Ns3dCtrl* ctrl;
  const T* lam;        // lambda_k by integer |k|^2 (evaluated in FP64 once), or null
  int form;            // 0: bh = F[u_j u_l] (6); 1: bh = F[(u.grad)u], 2: bh = F[u x omega] (3)
};

template <typename T> NS3D_HD T ctrl_dt(const Ns3dCtrl& c);
template <> NS3D_HD float ctrl_dt<float>(const Ns3dCtrl& c) { return c.dtf; }
template <> NS3D_HD double ctrl_dt<double>(const Ns3dCtrl& c) { return c.dt; }

// One thread per (member m, kx, ky, kz); j = ky * h + kz indexes the plane.
template <typename T>
NS3D_HD void spectral_point(const SpecArgs<T>& a, int m, int kx, int j) {
  const SpecT<T>& sp = a.sp;
  const int h = a.h, N = a.N;
  const int kz = j % h;
  const int ky = j / h;
  const long long off = (long long)kx * N * h + j;
  const long long plane = (long long)N * N * h;
  const cplx<T>* u0 = a.u0 + m * a.m3 + off;
  cplx<T>* out = a.out + m * a.m3 + off;

  T dt = T(0);
  if (a.stage >= 1) {
    Ns3dCtrl& c = a.ctrl[m];
    dt = ctrl_dt<T>(c);
    if (!(dt > T(0))) {   // member finished: stages leave it unchanged
      if (out != u0)
        for (int q = 0; q < 3; ++q) out[q * plane] = u0[q * plane];
      if (a.stage == 3 && off == 0) c.umax_bits = 0ull;
      return;
    }
  }

  cplx<T> R[3];
  const int sx = kx < h ? kx : kx - N;
  const int sy = ky < h ? ky : ky - N;
  const int k2 = sx * sx + sy * sy + kz * kz;
  if (kx == h || ky == h || k2 == 0) {
    R[0] = R[1] = R[2] = czero<T>();
  } else {
    const cplx<T>* bh = a.bh + m * a.m6 + off;
    const T kx_ = sp.kscale * T(sx), ky_ = sp.kscale * T(sy), kz_ = sp.kscale * T(kz);
    cplx<T> bb[3];
    if (a.form == 0) {
      cplx<T> b6[6];
      for (int q = 0; q < 6; ++q) b6[q] = sp.inv_P3 * bh[q * plane];
      // kappa . B_j  (B symmetric: 00 01 02 11 12 22)
      const cplx<T> t0 = kx_ * b6[0] + ky_ * b6[1] + kz_ * b6[2];
      const cplx<T> t1 = kx_ * b6[1] + ky_ * b6[3] + kz_ * b6[4];
      const cplx<T> t2 = kx_ * b6[2] + ky_ * b6[4] + kz_ * b6[5];
      // b = -i t
      bb[0] = cmake(t0.y, -t0.x);
      bb[1] = cmake(t1.y, -t1.x);
      bb[2] = cmake(t2.y, -t2.x);
    } else {
      const T sg = a.form == 1 ? -sp.inv_P3 : sp.inv_P3;
      for (int q = 0; q < 3; ++q) bb[q] = sg * bh[q * plane];
    }
    const T kap2 = kx_ * kx_ + ky_ * ky_ + kz_ * kz_;
    const cplx<T> kb = (T(1) / kap2) * (kx_ * bb[0] + ky_ * bb[1] + kz_ * bb[2]);
    const T lam = a.lam ? a.lam[k2] : lambda_k<T>(k2, sp);
    // the dissipation acts on the field R is evaluated at: u_n at stages 0
    // and 1, the stage state at stages 2 and 3
    const cplx<T>* ue = (a.stage >= 2) ? a.us + m * a.m3 + off : u0;
    R[0] = bb[0] - kx_ * kb - lam * ue[0];
    R[1] = bb[1] - ky_ * kb - lam * ue[plane];
    R[2] = bb[2] - kz_ * kb - lam * ue[2 * plane];
  }

  for (int q = 0; q < 3; ++q) {
    const cplx<T> uj = u0[q * plane];
    cplx<T> v;
    if (a.stage == 0) v = R[q];
    else if (a.stage == 1) v = uj + dt * R[q];
    else {
      const cplx<T> w = a.us[m * a.m3 + off + q * plane] + dt * R[q];
      if (a.stage == 2) v = T(0.75) * uj + T(0.25) * w;
      else v = T(1.0 / 3.0) * uj + T(2.0 / 3.0) * w;
    }
    if (kx == h || ky == h) v = czero<T>();
    out[q * plane] = v;
  }
  if (a.stage == 3 && off == 0) {
    Ns3dCtrl& c = a.ctrl[m];
    c.t += c.dt;
    c.nsteps += 1;
    c.umax_bits = 0ull;
  }
}

// =====================================================================
// Writers' statistics (section 2.4; Algorithm 1 step 3).
// =====================================================================

// round(|k|) for an integer |k|^2: the K with (2K - 1)^2 <= 4 k2 < (2K + 1)^2
NS3D_HD int shell_of(int k2) {
  int K = (int)sqrtf((float)k2);
  while ((2 * K + 1) * (2 * K + 1) <= 4 * k2) ++K;
  while (K > 0 && (2 * K - 1) * (2 * K - 1) > 4 * k2) --K;
  return K;
}

// Inverse z pass without products: c2r of the three components of a tile
// of y columns to the physical grid u[c][x][y][z] (real, z contiguous).
template <typename T>
struct ZInvArgs {
  const cplx<T>* in;   // [3][x N][y N][kz h]
  T* out;              // [3][x N][y N][z N]
  const cplx<T>* tw;
  FftPlanDev pl;       // length N
  int N, h, W, ldw;
};

template <typename T, class Sync>
NS3D_HD void zinv_block(const ZInvArgs<T>& a, int bx, int by, int tid, int nthr, cplx<T>* sm,
                        const Sync& sync) {
  const int N = a.N, h = a.h, W = a.W, ldw = a.ldw;
  const int y0 = bx * W;
  const int ncol = imin(W, N - y0);
  const int half = W / 2;
  cplx<T>* U01 = sm;
  cplx<T>* U2 = sm + N * ldw;
  cplx<T>* A = sm + 2 * N * ldw;
  cplx<T>* B = sm + 3 * N * ldw;
  const long long cstride = (long long)N * N * h;
  const cplx<T>* in = a.in + by * (long long)N * h + (long long)y0 * h;
  SmemIO<T> u01{U01, ldw}, u2s{U2, ldw};
  ZLoadInv<T> l01{in, in + cstride, N, h, ncol, 0};
  fft_tile<T, +1, false, true>(a.pl, ncol, tid, nthr, a.tw, l01, u01, A, B, ldw, sync);
  sync();
  ZLoadInv<T> l22{in + 2 * cstride, in + 2 * cstride, N, h, ncol, half};
  fft_tile<T, +1, false, true>(a.pl, half, tid, nthr, a.tw, l22, u2s, A, B, ldw, sync);
  sync();
  ZPhys<T> ph{U01, U2, ldw, half};
  const long long N3 = (long long)N * N * N;
  T* out = a.out + (long long)by * N * N + (long long)y0 * N;
  for (int w = tid; w < N * ncol; w += nthr) {
    const int p = w % N, col = w / N;
    T u0, u1, u2;
    ph.get(col, p, u0, u1, u2);
    out[col * N + p] = u0;
    out[N3 + col * N + p] = u1;
    out[2 * N3 + col * N + p] = u2;
  }
}

// Welford update of the pointwise mean and co-moments with the n-th sample:
// mean_i += d_i / n, C_ij += d_i (x_j - mean_j_new), d = x - mean_old.
// C is stored for (i <= j) in the order 00 01 02 11 12 22.
template <typename T>
NS3D_HD void welford_point(const T* u, long long N3, long long i, int n, double* mean, double* C) {
  double x[3], d[3], e[3];
  for (int c = 0; c < 3; ++c) {
    x[c] = (double)u[c * N3 + i];
    d[c] = x[c] - mean[c * N3 + i];
    mean[c * N3 + i] += d[c] / n;
    e[c] = x[c] - mean[c * N3 + i];
  }
  int q = 0;
  for (int r = 0; r < 3; ++r)
    for (int s = r; s < 3; ++s, ++q) C[q * N3 + i] += d[r] * e[s];
}

// =====================================================================
// Discrete adjoint (not in the paper): the transpose of the linearised RHS,
//   J(u)^T w = T_N F[ sum_l u_l S_jl ] - lambda w,
//   S_jl = i kappa_l w'_j + i kappa_j w'_l,  w' = Leray(w),
// in the real inner product over the full spectrum.
// =====================================================================

// S_jl (order 00 01 02 11 12 22) of w' = Leray(w), one stored mode.
template <typename T>
NS3D_HD void adj_prep_point(const cplx<T>* w, cplx<T>* S6, int N, T kscale, int kx, int j) {
  const int h = N / 2;
  const int kz = j % h, ky = j / h;
  const long long plane = (long long)N * N * h;
  const long long off = (long long)kx * N * h + j;
  const int sx = kx < h ? kx : kx - N;
  const int sy = ky < h ? ky : ky - N;
  const T k[3] = {kscale * T(sx), kscale * T(sy), kscale * T(kz)};
  const T kap2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
  cplx<T> wp[3];
  if (kx == h || ky == h || kap2 == T(0)) {
    wp[0] = wp[1] = wp[2] = czero<T>();
  } else {
    const cplx<T> w0 = w[off], w1 = w[plane + off], w2 = w[2 * plane + off];
    const cplx<T> kw = (T(1) / kap2) * (k[0] * w0 + k[1] * w1 + k[2] * w2);
    wp[0] = w0 - k[0] * kw;
    wp[1] = w1 - k[1] * kw;
    wp[2] = w2 - k[2] * kw;
  }
  int q = 0;
  for (int r = 0; r < 3; ++r)
    for (int s = r; s < 3; ++s, ++q) {
      const cplx<T> t = k[s] * wp[r] + k[r] * wp[s];       // times i:
      S6[q * plane + off] = cmake(-t.y, t.x);
    }
}

// out = alpha w + beta dt (J^T w) + gamma X + delta Y at one stored mode, with
// J^T w = bh / P^3 - lambda w (bh the truncated forward transform of the
// products); Nyquist rows are zero.
template <typename T>
struct AdjCombineArgs {
  const cplx<T>* bh;
  const cplx<T>* w;
  const cplx<T>* X;
  const cplx<T>* Y;
  cplx<T>* out;
  int N;
  SpecT<T> sp;
  T dt, alpha, beta, gamma, delta;
};

template <typename T>
NS3D_HD void adj_combine_point(const AdjCombineArgs<T>& a, int kx, int j) {
  const int N = a.N, h = N / 2;
  const int kz = j % h, ky = j / h;
  const long long plane = (long long)N * N * h;
  const long long off = (long long)kx * N * h + j;
  const int sx = kx < h ? kx : kx - N;
  const int sy = ky < h ? ky : ky - N;
  const bool nyq = (kx == h || ky == h);
  const T lam = lambda_k<T>(sx * sx + sy * sy + kz * kz, a.sp);
  for (int c = 0; c < 3; ++c) {
    const long long i = c * plane + off;
    cplx<T> v = czero<T>();
    if (!nyq) {
      const cplx<T> jt = a.sp.inv_P3 * a.bh[i] - lam * a.w[i];
      v = a.alpha * a.w[i] + (a.beta * a.dt) * jt;
      if (a.X) v = v + a.gamma * a.X[i];
      if (a.Y) v = v + a.delta * a.Y[i];
    }
    a.out[i] = v;
  }
}

// Band mask: out = u where k_lo <= |k| < k_hi (|k| of the integer wavenumber)
template <typename T>
NS3D_HD void band_point(const cplx<T>* u, cplx<T>* out, int N, double k_lo, double k_hi, int kx, int j) {
  const int h = N / 2;
  const int kz = j % h, ky = j / h;
  const long long plane = (long long)N * N * h;
  const long long off = (long long)kx * N * h + j;
  const int sx = kx < h ? kx : kx - N;
  const int sy = ky < h ? ky : ky - N;
  const double km = sqrt((double)(sx * sx + sy * sy + kz * kz));
  const bool in = km >= k_lo && km < k_hi && kx != h && ky != h;
  for (int c = 0; c < 3; ++c) out[c * plane + off] = in ? u[c * plane + off] : czero<T>();
}

// Adjoint z pass: c2r of u (3) and S (6) packed as five complex lines per
// column -- (u0,u1) (u2,S00) (S01,S02) (S11,S12) (S22,0) -- the products
// c_j = sum_l u_l S_jl, and r2c of (c0,c1) and (c2,0), truncated.
template <typename T>
struct ZAdjArgs {
  const cplx<T>* in;   // [9][x P][y P][kz h]
  cplx<T>* out;        // [3][x P][y P][kz h]
  const cplx<T>* tw;
  FftPlanDev pl;
  int P, h, W, ldw;
};

template <typename T>
struct ZAdjLoadProd {
  const cplx<T>* U[5];
  int ldw, line;   // line 0: c0 + i c1, line 1: c2
  NS3D_HD cplx<T> operator()(int col, int p) const {
    const int o = p * ldw + col;
    const cplx<T> a = U[0][o], b = U[1][o], c = U[2][o], d = U[3][o], e = U[4][o];
    const T u0 = a.x, u1 = a.y, u2 = b.x;
    const T S00 = b.y, S01 = c.x, S02 = c.y, S11 = d.x, S12 = d.y, S22 = e.x;
    if (line == 0) return cmake(u0 * S00 + u1 * S01 + u2 * S02, u0 * S01 + u1 * S11 + u2 * S12);
    return cmake(u0 * S02 + u1 * S12 + u2 * S22, T(0));
  }
};

template <typename T, class Sync>
NS3D_HD void zadj_block(const ZAdjArgs<T>& a, int bx, int by, int tid, int nthr, cplx<T>* sm,
                        const Sync& sync) {
  const int P = a.P, h = a.h, W = a.W, ldw = a.ldw;
  const int y0 = bx * W;
  const int ncol = imin(W, P - y0);
  const long long cs = (long long)P * P * h;
  const cplx<T>* in = a.in + by * (long long)P * h + (long long)y0 * h;
  cplx<T>* U[5];
  for (int l = 0; l < 5; ++l) U[l] = sm + l * P * ldw;
  cplx<T>* A = sm + 5 * P * ldw;
  cplx<T>* B = sm + 6 * P * ldw;
  const int big = 1 << 30;
  for (int l = 0; l < 5; ++l) {
    const cplx<T>* ia = in + (2 * l) * cs;
    const cplx<T>* ib = in + (l < 4 ? 2 * l + 1 : 2 * l) * cs;
    ZLoadInvCols<T> ld{ia, ib, P, h, ncol, l < 4 ? 0 : big};
    SmemIO<T> st{U[l], ldw};
    fft_tile<T, +1, false, true>(a.pl, ncol, tid, nthr, a.tw, ld, st, A, B, ldw, sync);
    sync();
  }
  cplx<T>* out = a.out + by * (long long)P * h + (long long)y0 * h;
  for (int line = 0; line < 2; ++line) {
    ZAdjLoadProd<T> lp{{U[0], U[1], U[2], U[3], U[4]}, ldw, line};
    cplx<T>* E = fft_free_buffer(a.pl.npass, A, B);
    SmemIO<T> e{E, ldw};
    fft_tile<T, -1, true, true>(a.pl, ncol, tid, nthr, a.tw, lp, e, A, B, ldw, sync);
    sync();
    for (int w = tid; w < h * ncol; w += nthr) {
      const int k = w % h, col = w / h;
      const cplx<T> zk = E[k * ldw + col];
      const cplx<T> zm = cconj(E[((P - k) % P) * ldw + col]);
      const cplx<T> s = zk + zm, d = zk - zm;
      if (line == 0) {
        out[col * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
        out[cs + col * h + k] = cmake(T(0.5) * d.y, T(-0.5) * d.x);
      } else {
        out[2 * cs + col * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
      }
    }
    sync();
  }
}
