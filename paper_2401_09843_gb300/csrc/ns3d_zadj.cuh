// Register-resident z passes whose three products are sums over the lines of
// a column: the adjoint right-hand side (KIND 0) and the advective form of the
// nonlinear term (KIND 1), FP32, for the padded sizes of the forward register
// kernel (P = N1 * N2 in NS3D_FOR_ZFAST, default padding h = P/3).
//
// KIND 1 computes what zform_block computes for nonlinear_form = 1: from the
// inverse transforms of u and its nine derivatives, packed as (u0, u1),
// (u2, d0u0), (d1u0, d2u0), (d0u1, d1u1), (d2u1, d0u2), (d1u2, d2u2), the
// products N_j = sum_l u_l d_l u_j (N0, N1 complete after lines 2 and 4, N2
// after line 5), with the CFL maximum of |u0| + |u1| + |u2| and the
// finiteness test once u is complete; the forward lines are N0 + i N1 and N2.
// KIND 0 is described below.
//
// Same arithmetic as zadj_block (the transpose of the linearised nonlinear
// term: c2r of u and of the symmetric S = sym grad of the projected adjoint
// field, c_j = sum_l u_l S_jl at every point, r2c truncated to kz < N/2), on
// the plan of the rotational kernel (ns3d_zrot.cuh): one y column per slot,
// each transform one trip through shared memory.
//
//   inverse, pass 1   radix N1 from global memory; the slot's five lines pack
//                     the nine fields u0 u1 u2 S00 S01 S02 S11 S12 S22 two by
//                     two: (u0, u1), (u2, S00), (S01, S02), (S11, S12), (S22, 0)
//   inverse, pass 2   radix N2, line by line; thread (g, k1) keeps u and the
//                     running c at positions k1 + N1 k2 in registers:
//                       line 0  u0, u1
//                       line 1  u2;        c0  = u0 S00
//                       line 2  c0 += u1 S01 + u2 S02;  c1 = u0 S01;  c2 = u0 S02
//                       line 3  c1 += u1 S11 + u2 S12;  c2 += u1 S12
//                       line 4  c2 += u2 S22
//   forward, pass 1   radix N2 over the same positions: c0 + i c1 and c2
//   forward, pass 2   radix N1 in place
//   extraction        c0, c1 from the first line, c2 from the second
//
// The inverse lines go through shared memory in two parts, lines 0-2 and then
// lines 3 to NL - 1 (pass 1 of a part, barrier, pass 2 of that part, barrier),
// so that the exchange buffer holds three lines per column instead of NL:
// with the smaller buffer four CTAs fit on an SM instead of three (adjoint) or
// two (advective).
#pragma once

#include "ns3d_zfast.cuh"

// KIND 0: the adjoint's products (five inverse lines); KIND 1: the advective
// form's N_j = sum_l u_l d_l u_j (six inverse lines, nonlinear_form = 1)
template <int N1, int N2, int KIND = 0>
struct ZAdjShape {
  static constexpr int P = N1 * N2;
  static constexpr int H = P / 3;                      // N/2 of the default padding
  static constexpr int NSLOT = (N1 >= 24) ? 4 : 8;     // columns per CTA
  static constexpr int NTHR = NSLOT * N1;
  static constexpr int Y = NSLOT;
  static constexpr int NL = KIND == 1 ? 6 : 5;         // inverse lines per column
  static constexpr int NLA = 3;                        // lines of the first part
  static constexpr int NLR = 3;                        // exchange lines per column
  static constexpr int LP = P + (N1 > N2 ? N1 : N2);   // padded exchange rows
  static constexpr int SM_ELEMS = 2 * P + NSLOT * NLR * LP;
  static_assert(NL - NLA <= NLR && NLA <= NLR && NLR >= 2, "exchange lines");
};

template <typename T, int N1, int N2>
struct ZAdjState {
  cplx<T> u01[N2];   // (u0, u1)
  T u2[N2];
  cplx<T> c01[N2];   // (c0, c1), the first forward line
  T c2[N2];
  T umax;            // KIND 1: max of |u0| + |u1| + |u2| over the thread's points
  int bad;           // KIND 1: a non-finite value was seen
};

template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD ZFastCtx<T, N1, N2> zadjf_ctx(const ZArgs<T>& a, int bx, int by, int bz, cplx<T>* sm) {
  using S = ZAdjShape<N1, N2, KIND>;
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

// exchange row of line l of slot g (the two parts share the rows)
template <int N1, int N2, int KIND>
NS3D_HD int zadjf_row(int g, int l) {
  using S = ZAdjShape<N1, N2, KIND>;
  return (g * S::NLR + (l < S::NLA ? l : l - S::NLA)) * S::LP;
}

// inverse pass 1 of part `part` (lines 0..NLA-1, or NLA..NL-1): tasks (slot g,
// line l, j2), j2 fastest; line l packs fields 2l and 2l + 1 of column y0 + g
// (line 4: field 8 and zero)
template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD void zadjf_inv1(const ZFastCtx<T, N1, N2>& c, int tid, int nthr, int part) {
  using S = ZAdjShape<N1, N2, KIND>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  constexpr bool full = (S::P % S::Y == 0);     // every tile has Y columns
  const cplx<T>* in = a.in + c.bz * a.in_bs + c.by * a.xs + (long long)c.y0 * h;
  const int l0 = part ? S::NLA : 0, nl = part ? S::NL - S::NLA : S::NLA;
  for (int t = tid; t < S::NSLOT * nl * N2; t += nthr) {
    const int j2 = t % N2;
    const int l = l0 + (t / N2) % nl;
    const int g = t / (nl * N2);
    int fa = 2 * l, fb = l < 4 ? 2 * l + 1 : -1;  // adjoint: the last line has one field
    if (KIND == 1) form_pair(1, l, &fa, &fb);      // advective: the zform packing
    const bool two = fb >= 0;
    const cplx<T>* ia = in + fa * a.in_cs;
    const cplx<T>* ib = in + (two ? fb : fa) * a.in_cs;
    cplx<T> v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int p = N2 * j1 + j2;
      const int reg = pad_region(N2 * j1, N2, S::P, S::H);
      if (reg == PAD_ZERO) {
        v[j1] = czero<T>();
      } else if (full && reg == PAD_LOW) {          // a[p] + i b[p]
        cplx<T> x = ia[g * h + p], y = two ? ib[g * h + p] : czero<T>();
        if (j1 == 0 && p == 0) {                    // real lines have a real mean
          x.y = T(0);
          y.y = T(0);
        }
        v[j1] = cmake(x.x - y.y, x.y + y.x);
      } else if (full && reg == PAD_HIGH) {         // conj(a[P-p]) + i conj(b[P-p])
        const cplx<T> x = ia[g * h + (S::P - p)], y = two ? ib[g * h + (S::P - p)] : czero<T>();
        v[j1] = cmake(x.x + y.y, -x.y + y.x);
      } else {
        v[j1] = pack2(ia, two ? ib : ia, S::P, S::H, p, g, two ? g : S::P, c.ncol);
      }
    }
    Dft<N1, +1>::run(v);
    cplx<T>* X = c.X + zadjf_row<N1, N2, KIND>(g, l);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1)
      X[j2 * (N1 + 1) + k1] = k1 == 0 ? v[k1] : v[k1] * c.twi[k1 * N2 + j2];
  }
}

// inverse pass 2 of line l into v (positions k1 + N1 k2 of slot g)
template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD void zadjf_line(const ZFastCtx<T, N1, N2>& c, int g, int k1, int l, cplx<T>* v) {
  const cplx<T>* X = c.X + zadjf_row<N1, N2, KIND>(g, l);
#pragma unroll
  for (int j = 0; j < N2; ++j) v[j] = X[j * (N1 + 1) + k1];
  Dft<N2, +1>::run(v);
}

// inverse pass 2 of the lines of part `part` and the products c_j = sum_l u_l S_jl
template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD void zadjf_inv2(const ZFastCtx<T, N1, N2>& c, int tid, ZAdjState<T, N1, N2>& st, int part) {
  const int k1 = tid % N1;
  const int g = tid / N1;
  cplx<T> v[N2];
  if (KIND == 1 && part == 1) {
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 3, v);                      // (d0 u1, d1 u1)
#pragma unroll
    for (int k = 0; k < N2; ++k) st.c01[k].y = st.u01[k].x * v[k].x + st.u01[k].y * v[k].y;
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 4, v);                      // (d2 u1, d0 u2)
#pragma unroll
    for (int k = 0; k < N2; ++k) {
      st.c01[k].y = st.c01[k].y + st.u2[k] * v[k].x;
      st.c2[k] = st.u01[k].x * v[k].y;
    }
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 5, v);                      // (d1 u2, d2 u2)
#pragma unroll
    for (int k = 0; k < N2; ++k) st.c2[k] = st.c2[k] + st.u01[k].y * v[k].x + st.u2[k] * v[k].y;
    return;
  }
  if (KIND == 0 && part == 1) {
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 3, v);                      // (S11, S12)
#pragma unroll
    for (int k = 0; k < N2; ++k) {
      const T u1 = st.u01[k].y, u2 = st.u2[k];
      st.c01[k].y = st.c01[k].y + u1 * v[k].x + u2 * v[k].y;
      st.c2[k] = st.c2[k] + u1 * v[k].y;
    }
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 4, v);                      // (S22, 0)
#pragma unroll
    for (int k = 0; k < N2; ++k) st.c2[k] = st.c2[k] + st.u2[k] * v[k].x;
    return;
  }
  zadjf_line<T, N1, N2, KIND>(c, g, k1, 0, st.u01);
  if (KIND == 1) {   // advective: N_j = sum_l u_l d_l u_j into c01 = (N0, N1), c2 = N2
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 1, v);                      // (u2, d0 u0)
    using S = ZAdjShape<N1, N2, KIND>;
    constexpr bool full = S::P % S::Y == 0;
    const bool valid = full || g < c.ncol;
    T m = T(0), chk = T(0);   // 0 * s is 0 exactly when s is finite; the maximum skips NaN
#pragma unroll
    for (int k = 0; k < N2; ++k) {
      st.u2[k] = v[k].x;
      st.c01[k] = cmake(st.u01[k].x * v[k].y, T(0));
      const T sum = xabs(st.u01[k].x) + xabs(st.u01[k].y) + xabs(v[k].x);
      if (valid) {
        m = xmax(m, sum);
        chk = chk + T(0) * sum;
      }
    }
    st.bad = !(chk == T(0)) || !(m <= big_finite<T>());
    st.umax = m;
    zadjf_line<T, N1, N2, KIND>(c, g, k1, 2, v);                      // (d1 u0, d2 u0)
#pragma unroll
    for (int k = 0; k < N2; ++k)
      st.c01[k].x = st.c01[k].x + st.u01[k].y * v[k].x + st.u2[k] * v[k].y;
    return;
  }
  zadjf_line<T, N1, N2, KIND>(c, g, k1, 1, v);                        // (u2, S00)
#pragma unroll
  for (int k = 0; k < N2; ++k) {
    st.u2[k] = v[k].x;
    st.c01[k] = cmake(st.u01[k].x * v[k].y, T(0));
  }
  zadjf_line<T, N1, N2, KIND>(c, g, k1, 2, v);                        // (S01, S02)
#pragma unroll
  for (int k = 0; k < N2; ++k) {
    const T u0 = st.u01[k].x, u1 = st.u01[k].y, u2 = st.u2[k];
    st.c01[k] = cmake(st.c01[k].x + u1 * v[k].x + u2 * v[k].y, u0 * v[k].x);
    st.c2[k] = u0 * v[k].y;
  }
}

// forward pass 1: radix N2 over the thread's own positions, two lines
template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD void zadjf_fwd1(const ZFastCtx<T, N1, N2>& c, int tid, const ZAdjState<T, N1, N2>& st) {
  using S = ZAdjShape<N1, N2, KIND>;
  const int k1 = tid % N1;
  const int g = tid / N1;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    cplx<T> v[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = q == 0 ? st.c01[k2] : cmake(st.c2[k2], T(0));
    Dft<N2, -1>::run(v);
    cplx<T>* X = c.X + (g * S::NLR + q) * S::LP;
#pragma unroll
    for (int k = 0; k < N2; ++k)
      X[k1 * (N2 + 1) + k] = k == 0 ? v[k] : v[k] * c.twf[k * N1 + k1];
  }
}

// forward pass 2: radix N1 in place; tasks (g, q < 2, kappa < N2)
template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD void zadjf_fwd2(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZAdjShape<N1, N2, KIND>;
  for (int t = tid; t < S::NSLOT * 2 * N2; t += nthr) {
    const int kap = t % N2;
    const int lq = t / N2;
    cplx<T>* X = c.X + ((lq >> 1) * S::NLR + (lq & 1)) * S::LP;
    cplx<T> v[N1];
#pragma unroll
    for (int q = 0; q < N1; ++q) v[q] = X[q * (N2 + 1) + kap];
    Dft<N1, -1>::run(v);
#pragma unroll
    for (int k = 0; k < N1; ++k)   // position kap + N2 k; the truncated band is never read
      if (pad_region(N2 * k, N2, S::P, S::H) != PAD_ZERO) X[k * (N2 + 1) + kap] = v[k];
  }
}

// extraction: kz < h of the real lines c0, c1 (first line) and c2 (second);
// tasks (g, q, k), k fastest so that a warp's stores are contiguous
template <typename T, int N1, int N2, int KIND = 0>
NS3D_HD void zadjf_extract(const ZFastCtx<T, N1, N2>& c, int tid, int nthr) {
  using S = ZAdjShape<N1, N2, KIND>;
  const ZArgs<T>& a = *c.a;
  constexpr int h = S::H;
  constexpr bool full = S::P % S::Y == 0;
  cplx<T>* out = a.out + c.bz * a.out_bs + c.by * a.xs + (long long)c.y0 * h;
  for (int t = tid; t < S::NSLOT * 2 * h; t += nthr) {
    const int k = t % h;
    const int lq = t / h;
    const int g = lq >> 1, q = lq & 1;
    if (!full && g >= c.ncol) continue;
    const cplx<T>* X = c.X + (g * S::NLR + q) * S::LP;
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
