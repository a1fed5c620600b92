// Column pass with a three-pass register FFT, for long transforms
// P = N1 * N2 * N3 (P = 1536 = 16 * 12 * 8 at N = 1024) whose radices are
// all register codelets.
//
// Same contract as colfft_block and colfast (1D transforms along one axis of
// a strided array, padding on load for the inverse, truncation on store for
// the forward; Algorithm 3 steps 1-2 and their reverse).  With input index
// j = N2 N3 j1 + N3 j2 + j3 and output index k = k1 + N1 k2 + N1 N2 k3:
//
//   pass 1  task (column c, j' = N3 j2 + j3): radix N1 over x[N2 N3 j1 + j']
//           loaded from global memory (a warp reads 16 adjacent columns of a
//           row; blocks of the zero band known at compile time are not
//           loaded), twiddle w_P^(j' k1), to D[c][j' N1 + k1]
//   pass 2  task (c, k1, j3): radix N2 over D[c][(N3 j2 + j3) N1 + k1],
//           twiddle w_P^(N1 j3 k2) (= w_{N2 N3}^(j3 k2)), written back to the
//           slots it read (k2 in place of j2): no barrier between its reads
//           and writes
//   pass 3  task (c, k1, k2): radix N3 over D[c][(N3 k2 + j3) N1 + k1], result
//           X[k1 + N1 k2 + N1 N2 k3] to global memory (blocks of the
//           truncated band known at compile time are not stored)
//
// One shared line of P + 1 elements per column (odd stride: the 16 columns a
// warp touches fall in distinct banks).  Storage type T (global memory),
// arithmetic type C = LongC<T> (registers and shared memory): FP64 data are
// transformed in double-single arithmetic (ns3d_df64.cuh).
#pragma once

#include "ns3d_blocks.cuh"
#include "ns3d_df64.cuh"

// Long transform lengths with a three-pass register column pass (FP32),
// used with the default padding h = N/2 = P/3.
#define NS3D_FOR_COLFAST3(X) X(16, 12, 8)

// ESZ: bytes of one complex element (8 FP32, 16 FP64)
template <int N1, int N2, int N3, int ESZ = 8>
struct ColFast3Shape {
  static constexpr int P = N1 * N2 * N3;
  static constexpr int H = P / 3;        // N/2 of the default padding P = 3N/2
  // columns per CTA: 16, or 8 where 16 lines would not fit in shared memory
  static constexpr int W = (P + 16 * (P + 1)) * ESZ <= 220 * 1024 ? 16 : 8;
  static constexpr int NTHR = 512;
  static constexpr int LP = P + 1;
  static constexpr int SM_ELEMS = P + W * LP;
};

template <typename T, int SIGN, int P>
NS3D_HD void colfast3_twiddles(cplx<LongC<T>>* tw, const cplx<T>* gtw, int tid, int nthr) {
  for (int e = tid; e < P; e += nthr) {
    cplx<T> w = gtw[e];
    if (SIGN > 0) w.y = -w.y;
    tw[e] = ccvt<LongC<T>>(w);
  }
}

// PAD: the input has N = 2H rows spread over the P positions (inverse).
template <typename T, int SIGN, int N1, int N2, int N3, bool PAD>
NS3D_HD void colfast3_pass1(const ColArgs<T>& a, int bx, int by, int bz, int tid, int nthr,
                            const cplx<LongC<T>>* tw, cplx<LongC<T>>* X) {
  using S = ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>;
  using C = LongC<T>;
  constexpr int M = N2 * N3;
  const int c0 = bx * S::W;
  const int ncol = imin(S::W, a.ncols - c0);
  const cplx<T>* in = a.in + bz * a.in_bs + by * a.in_os + c0 * a.in_cs;
#pragma unroll 1
  for (int t = tid; t < S::W * M; t += nthr) {
    const int col = t % S::W;
    const int jp = t / S::W;
    if (col >= ncol) continue;
    const cplx<T>* ic = in + col * a.in_cs;
    const int rs = (int)a.in_rs;   // P rs < 2^31 (checked at dispatch)
    cplx<C> v[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int p = M * j1 + jp;
      if (!PAD) {
        v[j1] = ccvt<C>(ic[p * rs]);
      } else {
        const int reg = pad_region(M * j1, M, S::P, S::H);
        if (reg == PAD_ZERO) {
          v[j1] = czero<C>();
        } else if (reg == PAD_LOW) {
          v[j1] = ccvt<C>(ic[p * rs]);
        } else if (reg == PAD_HIGH) {
          v[j1] = ccvt<C>(ic[(p - S::H) * rs]);   // row p - P + N
        } else {
          const int row = pad_row_of(p, S::P, S::H, 2 * S::H);
          v[j1] = row >= 0 ? ccvt<C>(ic[row * rs]) : czero<C>();
        }
      }
    }
    Dft<N1, SIGN>::run(v);
    cplx<C>* D = X + col * S::LP + jp * N1;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) D[k1] = k1 == 0 ? v[k1] : v[k1] * tw[jp * k1];   // tw[0] = 1
  }
}

template <typename T, int SIGN, int N1, int N2, int N3>
NS3D_HD void colfast3_pass2(int tid, int nthr, int ncol, const cplx<LongC<T>>* tw,
                            cplx<LongC<T>>* X) {
  using S = ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>;
  using C = LongC<T>;
#pragma unroll 1
  for (int t = tid; t < S::W * N1 * N3; t += nthr) {
    const int col = t % S::W;
    const int r = t / S::W;
    const int k1 = r % N1, j3 = r / N1;
    if (col >= ncol) continue;
    cplx<C>* D = X + col * S::LP + j3 * N1 + k1;
    cplx<C> v[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) v[j2] = D[j2 * N3 * N1];
    Dft<N2, SIGN>::run(v);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) D[k2 * N3 * N1] = k2 == 0 ? v[k2] : v[k2] * tw[N1 * j3 * k2];
  }
}

// TRUNC: only the N = 2H retained positions are stored (forward).
template <typename T, int SIGN, int N1, int N2, int N3, bool TRUNC>
NS3D_HD void colfast3_pass3(const ColArgs<T>& a, int bx, int by, int bz, int tid, int nthr,
                            const cplx<LongC<T>>* X) {
  using S = ColFast3Shape<N1, N2, N3, (int)sizeof(cplx<T>)>;
  using C = LongC<T>;
  const C scale = (C)a.scale;
  constexpr int M = N1 * N2;
  const int c0 = bx * S::W;
  const int ncol = imin(S::W, a.ncols - c0);
  cplx<T>* out = a.out + bz * a.out_bs + by * a.out_os + c0 * a.out_cs;
#pragma unroll 1
  for (int t = tid; t < S::W * M; t += nthr) {
    const int col = t % S::W;
    const int r = t / S::W;
    const int k1 = r % N1, k2 = r / N1;
    if (col >= ncol) continue;
    const cplx<C>* D = X + col * S::LP + k2 * N3 * N1 + k1;
    cplx<C> v[N3];
#pragma unroll
    for (int j3 = 0; j3 < N3; ++j3) v[j3] = D[j3 * N1];
    Dft<N3, SIGN>::run(v);
    cplx<T>* oc = out + col * a.out_cs;
    const int rs = (int)a.out_rs;  // P rs < 2^31 (checked at dispatch)
#pragma unroll
    for (int k3 = 0; k3 < N3; ++k3) {
      const int p = r + M * k3;
      if (!TRUNC) {
        oc[p * rs] = ccvt<T>(scale * v[k3]);
      } else {
        const int reg = pad_region(M * k3, M, S::P, S::H);
        if (reg == PAD_LOW) {
          oc[p * rs] = ccvt<T>(scale * v[k3]);
        } else if (reg == PAD_HIGH) {
          oc[(p - S::H) * rs] = ccvt<T>(scale * v[k3]);
        } else if (reg == PAD_MIXED) {
          const int row = pad_row_of(p, S::P, S::H, 2 * S::H);
          if (row >= 0) oc[row * rs] = ccvt<T>(scale * v[k3]);
        }
      }
    }
  }
  if (TRUNC)   // the Nyquist row N/2 receives no position: keep it zero
    for (int col = tid; col < ncol; col += nthr) out[col * a.out_cs + S::H * a.out_rs] = czero<T>();
}
