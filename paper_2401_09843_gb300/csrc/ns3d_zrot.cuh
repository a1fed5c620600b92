// Register-resident z pass of the rotational form (nonlinear_form = 2), FP32,
// for the padded sizes of the divergence form's register kernel
// (P = N1 * N2 in NS3D_FOR_ZFAST, default padding h = P/3).
//
// Same plan as ns3d_zfast.cuh with one y column per slot instead of a pair of
// columns: a slot's three inverse lines are u0 + i u1, u2 + i w0 and w1 + i w2
// of its column (fields 0..5 of the form's input, w = curl u), the physical
// values stay in the thread's registers after the second inverse pass,
// p = u x w is formed there, and two forward lines, p0 + i p1 and p2 (real),
// are transformed and extracted: the first into output components 0 and 1,
// the second into component 2.  The thread state (three lines of N2 values)
// is the divergence kernel's.
#pragma once

#include "ns3d_zfast.cuh"

template <int N1, int N2>
struct ZRotShape {
  static constexpr int P = N1 * N2;
  static constexpr int H = P / 3;                      // N/2 of the default padding
  static constexpr int NSLOT = (N1 >= 24) ? 4 : 16;    // columns per CTA
  static constexpr int NTHR = NSLOT * N1;
  static constexpr int Y = NSLOT;
  static constexpr int LP = P + (N1 > N2 ? N1 : N2);   // padded exchange rows
  static constexpr int SM_ELEMS = 2 * P + NSLOT * 3 * LP;
};

template <typename T, int N1, int N2>
NS3D_HD ZFastCtx<T, N1, N2> zrot_ctx(const ZArgs<T>& a, int bx, int by, int bz, cplx<T>* sm) {
  using S = ZRotShape<N1, N2>;
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

// inverse pass 1: tasks (slot g, line l, j2), j2 fastest; line l packs fields
// 2l and 2l + 1 of column y0 + g
template <typename T, int N1, int N2>
NS3D_HD void zrot_inv1(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZRotShape<N1, N2>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  constexpr bool full = (S::P % S::Y == 0);     // every tile has Y columns
  const cplx<T>* in = a.in + c.bz * a.in_bs + c.by * a.xs + (long long)c.y0 * h;
  for (int t = tid; t < S::NSLOT * 3 * N2; t += nthr) {
    const int j2 = t % N2;
    const int l = (t / N2) % 3;
    const int g = t / (3 * N2);
    const cplx<T>* ia = in + (2 * l) * a.in_cs;
    const cplx<T>* ib = in + (2 * l + 1) * a.in_cs;
    cplx<T> v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int p = N2 * j1 + j2;
      const int reg = pad_region(N2 * j1, N2, S::P, S::H);
      if (reg == PAD_ZERO) {
        v[j1] = czero<T>();
      } else if (full && reg == PAD_LOW) {          // a[p] + i b[p]
        cplx<T> x = ia[g * h + p], y = ib[g * h + p];
        if (j1 == 0 && p == 0) {                    // real lines have a real mean
          x.y = T(0);
          y.y = T(0);
        }
        v[j1] = cmake(x.x - y.y, x.y + y.x);
      } else if (full && reg == PAD_HIGH) {         // conj(a[P-p]) + i conj(b[P-p])
        const cplx<T> x = ia[g * h + (S::P - p)], y = ib[g * h + (S::P - p)];
        v[j1] = cmake(x.x + y.y, -x.y + y.x);
      } else {
        v[j1] = pack2(ia, ib, S::P, S::H, p, g, g, c.ncol);
      }
    }
    Dft<N1, +1>::run(v);
    cplx<T>* X = c.X + (g * 3 + l) * S::LP;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      X[j2 * (N1 + 1) + k1] = k1 == 0 ? v[k1] : v[k1] * c.twi[k1 * N2 + j2];
  }
}

// inverse pass 2: thread (g, k1) keeps positions k1 + N1 k2 of its column's
// three lines; CFL maximum of |u0| + |u1| + |u2| and the finiteness test
template <typename T, int N1, int N2>
NS3D_HD void zrot_inv2(const ZFastCtx<T, N1, N2>& c, int tid, ZFastState<T, N1, N2>& st) {
  using S = ZRotShape<N1, N2>;
  const int k1 = tid % N1;
  const int g = tid / N1;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const cplx<T>* X = c.X + (g * 3 + l) * S::LP;
#pragma unroll
    for (int j = 0; j < N2; ++j) st.z[l][j] = X[j * (N1 + 1) + k1];
    Dft<N2, +1>::run(st.z[l]);
  }
  constexpr bool full = S::P % S::Y == 0;
  const bool valid = full || g < c.ncol;
  T m = T(0), chk = T(0);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    const T s = xabs(st.z[0][k2].x) + xabs(st.z[0][k2].y) + xabs(st.z[1][k2].x);
    if (valid) {
      m = xmax(m, s);
      chk = chk + T(0) * s;   // 0 exactly when s is finite
    }
  }
  st.bad = !(chk == T(0)) || !(m <= big_finite<T>());
  st.umax = m;
}

// forward line q of the slot at register position k2: q = 0 p0 + i p1,
// q = 1 p2, with p = u x w
template <typename T, int N1, int N2>
NS3D_HD cplx<T> zrot_product(const ZFastState<T, N1, N2>& st, int q, int k2) {
  const T u0 = st.z[0][k2].x, u1 = st.z[0][k2].y;
  const T u2 = st.z[1][k2].x, w0 = st.z[1][k2].y;
  const T w1 = st.z[2][k2].x, w2 = st.z[2][k2].y;
  if (q == 0) return cmake(u1 * w2 - u2 * w1, u2 * w0 - u0 * w2);
  return cmake(u0 * w1 - u1 * w0, T(0));
}

// forward pass 1: radix N2 over the thread's own positions, two lines
template <typename T, int N1, int N2>
NS3D_HD void zrot_fwd1(const ZFastCtx<T, N1, N2>& c, int tid, const ZFastState<T, N1, N2>& st) {
  using S = ZRotShape<N1, N2>;
  const int k1 = tid % N1;
  const int g = tid / N1;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    cplx<T> v[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = zrot_product<T, N1, N2>(st, q, k2);
    Dft<N2, -1>::run(v);
    cplx<T>* X = c.X + (g * 3 + q) * S::LP;
#pragma unroll
    for (int k = 0; k < N2; ++k)
      X[k1 * (N2 + 1) + k] = k == 0 ? v[k] : v[k] * c.twf[k * N1 + k1];
  }
}

// forward pass 2: radix N1 in place; tasks (g, q < 2, kappa < N2)
template <typename T, int N1, int N2>
NS3D_HD void zrot_fwd2(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZRotShape<N1, N2>;
  for (int t = tid; t < S::NSLOT * 2 * N2; t += nthr) {
    const int kap = t % N2;
    const int lq = t / N2;
    cplx<T>* X = c.X + ((lq >> 1) * 3 + (lq & 1)) * S::LP;
    cplx<T> v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = X[q * (N2 + 1) + kap];
    Dft<N1, -1>::run(v);
#pragma unroll
    for (int k = 0; k < N1; ++k)   // position kap + N2 k; the truncated band is never read
      if (pad_region(N2 * k, N2, S::P, S::H) != PAD_ZERO) X[k * (N2 + 1) + kap] = v[k];
  }
}

// extraction: kz < h of the real lines; tasks (g, q, k), k fastest so that
// the stores of a warp are contiguous
template <typename T, int N1, int N2>
NS3D_HD void zrot_extract(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZRotShape<N1, N2>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  constexpr bool full = S::P % S::Y == 0;
  cplx<T>* out = a.out + c.bz * a.out_bs + c.by * a.xs + (long long)c.y0 * h;
  for (int t = tid; t < S::NSLOT * 2 * h; t += nthr) {
    const int k = t % h;
    const int lq = t / h;
    const int g = lq >> 1, q = lq & 1;
    if (!full && g >= c.ncol) continue;
    const cplx<T>* X = c.X + (g * 3 + q) * S::LP;
    const cplx<T> zk = X[zfast_fpos<N1, N2>(k)];
    const cplx<T> zm = cconj(X[zfast_fpos<N1, N2>(k == 0 ? 0 : S::P - k)]);
    const cplx<T> s = zk + zm;
    if (q == 0) {
      const cplx<T> d = zk - zm;
      out[g * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
      out[a.out_cs + g * h + k] = cmake(T(0.5) * d.y, T(-0.5) * d.x);   // d / (2i)
    } else {
      out[2 * a.out_cs + g * h + k] = cmake(T(0.5) * s.x, T(0.5) * s.y);
    }
  }
}
