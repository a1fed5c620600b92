// Column pass with a two-pass register FFT, for transform lengths
// P = N1 * N2 with both radices in registers (P = 48, 96, 192, 384).
//
// Same contract as colfft_block (1D transforms along one axis of a strided
// array, padding on load for the inverse, truncation on store for the
// forward; Algorithm 3 steps 1-2 and their reverse), specialised so that the
// index arithmetic is compile-time and every transform makes one trip through
// shared memory:
//
//   pass 1  task (column c, j2 < N2): radix N1 over x[N2 j1 + j2] loaded from
//           global memory (column-fast: a warp reads 16 or 32 adjacent columns
//           of a row), twiddle w_P^(j2 k1), store D[c][j2 N1 + k1]
//   pass 2  task (c, k1 < N1): radix N2 over D[c][j N1 + k1], result
//           X[k1 + N1 k2] stored to global memory
//
// A column's line occupies P + 1 shared elements (odd stride: the 16 columns a
// warp touches fall in distinct banks).
#pragma once

#include "ns3d_blocks.cuh"

// Transform lengths with a register-resident column pass (FP32): P = N1 * N2,
// used with the default padding h = N/2 = P/3 (compile-time zero band).
#define NS3D_FOR_COLFAST(X) X(24, 16) X(12, 16) X(12, 8) X(6, 8)

template <int N1, int N2>
struct ColFastShape {
  static constexpr int P = N1 * N2;
  static constexpr int H = P / 3;        // N/2 of the default padding P = 3N/2
  // P = 96 (12 x 8): 32 columns and 128 threads, so that both passes have a
  // whole number of tasks per thread (2 and 3) and a warp reads 256 contiguous
  // bytes of a row; otherwise 16 columns
  static constexpr bool WIDE = N1 == 12 && N2 == 8;
  static constexpr int W = WIDE ? 32 : 16;   // columns per CTA
  // one pass-2 task per thread at radix 24 (36 warps per SM), else 256 (32 warps)
  static constexpr int NTHR = WIDE ? 128 : (N1 >= 24 ? 384 : 256);
  static constexpr int MINB = WIDE ? 8 : (N1 >= 24 ? 3 : 4);
  static constexpr int LP = P + 1;
  static constexpr int SM_ELEMS = P + W * LP;
};

template <typename T, int SIGN, int N1, int N2>
NS3D_HD void colfast_twiddles(cplx<T>* tw, const cplx<T>* gtw, int tid, int nthr) {
  for (int e = tid; e < N1 * N2; e += nthr) {
    cplx<T> w = gtw[e];
    if (SIGN > 0) w.y = -w.y;
    tw[e] = w;
  }
}

// PAD: the input has N = 2H rows spread over the P positions (inverse).
template <typename T, int SIGN, int N1, int N2, bool PAD>
NS3D_HD void colfast_pass1(const ColArgs<T>& a, int bx, int by, int bz, int tid, int nthr,
                           const cplx<T>* tw, cplx<T>* X) {
  using S = ColFastShape<N1, N2>;
  const int c0 = bx * S::W;
  const int ncol = imin(S::W, a.ncols - c0);
  const cplx<T>* in = a.in + bz * a.in_bs + by * a.in_os + c0 * a.in_cs;
  const int cs = (int)a.in_cs, rs = (int)a.in_rs;
  for (int t = tid; t < S::W * N2; t += nthr) {
    const int col = t % S::W;
    const int j2 = t / S::W;
    if (col >= ncol) continue;
    cplx<T> v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int p = N2 * j1 + j2;
      if (!PAD) {
        v[j1] = in[col * cs + p * rs];
      } else if (pad_region(N2 * j1, N2, S::P, S::H) == PAD_ZERO) {
        v[j1] = czero<T>();
      } else {
        const int row = pad_row_of(p, S::P, S::H, 2 * S::H);
        v[j1] = row >= 0 ? in[col * cs + row * rs] : czero<T>();
      }
    }
    Dft<N1, SIGN>::run(v);
    cplx<T>* D = X + col * S::LP + j2 * N1;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) D[k1] = (k1 == 0 || j2 == 0) ? v[k1] : v[k1] * tw[j2 * k1];
  }
}

// TRUNC: only the N = 2H retained positions are stored (forward).
template <typename T, int SIGN, int N1, int N2, bool TRUNC>
NS3D_HD void colfast_pass2(const ColArgs<T>& a, int bx, int by, int bz, int tid, int nthr,
                           const cplx<T>* X) {
  using S = ColFastShape<N1, N2>;
  const int c0 = bx * S::W;
  const int ncol = imin(S::W, a.ncols - c0);
  cplx<T>* out = a.out + bz * a.out_bs + by * a.out_os + c0 * a.out_cs;
  const int cs = (int)a.out_cs, rs = (int)a.out_rs;
  for (int t = tid; t < S::W * N1; t += nthr) {
    const int col = t % S::W;
    const int k1 = t / S::W;
    if (col >= ncol) continue;
    cplx<T> v[N2];
    const cplx<T>* D = X + col * S::LP + k1;
#pragma unroll
    for (int j = 0; j < N2; ++j) v[j] = D[j * N1];
    Dft<N2, SIGN>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int p = k1 + N1 * k2;
      if (!TRUNC) {
        out[col * cs + p * rs] = a.scale * v[k2];
      } else if (pad_region(N1 * k2, N1, S::P, S::H) != PAD_ZERO) {
        const int row = pad_row_of(p, S::P, S::H, 2 * S::H);
        if (row >= 0) out[col * cs + row * rs] = a.scale * v[k2];
      }
    }
  }
  if (TRUNC)   // the Nyquist row N/2 receives no position: keep it zero
    for (int col = tid; col < ncol; col += nthr) out[col * cs + S::H * rs] = czero<T>();
}
