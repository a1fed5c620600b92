// Tile FFT engine: batched 1D transforms of the columns of a tile held in
// shared memory, as a sequence of Stockham radix passes.
//
// A tile holds `ncol` independent lines ("columns") of length n.  Pass p with
// radix R works on D[j][kappa] (j < M = n/L remaining time index, kappa < L
// frequencies already resolved; flat index j*L + kappa):
//
//   for each column, kappa < L and jl < S = M/R:
//     v[q] = D[S q + jl][kappa]                          q = 0..R-1
//     v    = DFT_R(v)                                    (in registers)
//     v[k] *= w_M^(jl k),  w_M = exp(SIGN 2 pi i / M)    (skipped when S = 1)
//     D'[jl][kappa + L k] = v[k]                         (next L' = L R)
//
// Pass 1 (L = 1) reads the input x[j] = D[j][0] through a loader functor and
// the last pass (M = R, so S = 1) hands X[kappa + L k] to a store functor, so
// the first and last passes talk to global memory directly and only the
// passes in between go through shared memory.  The shared layout is
// [position][column] with a padded column count `ldw`: when the column index
// varies fastest across threads ("column-fast" mapping) consecutive threads
// touch consecutive addresses; when the pass index varies fastest
// ("task-fast", used where the global data is contiguous along the transform
// axis) the odd stride ldw keeps shared-memory banks distinct.
//
// Everything here is __host__ __device__: the same code is run on the CPU by
// the index-logic self test (fft_host_selftest) before it runs on a GPU.
#pragma once

#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define NS3D_HD __host__ __device__ __forceinline__
#define NS3D_HDC __host__ __device__ constexpr
#else
#define NS3D_HD inline
#define NS3D_HDC constexpr
#endif

template <typename T>
struct alignas(2 * sizeof(T)) cplx {
  T x, y;
};

template <typename T> NS3D_HD cplx<T> cmake(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <typename T> NS3D_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return cmake(a.x + b.x, a.y + b.y); }
template <typename T> NS3D_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return cmake(a.x - b.x, a.y - b.y); }
template <typename T> NS3D_HD cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return cmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> NS3D_HD cplx<T> operator*(T s, cplx<T> a) { return cmake(s * a.x, s * a.y); }
template <typename T> NS3D_HD cplx<T> cconj(cplx<T> a) { return cmake(a.x, -a.y); }
template <typename T> NS3D_HD cplx<T> czero() { return cmake(T(0), T(0)); }

#include "codelets.cuh"

#define NS3D_MAX_PASSES 8

// Radix plan of one transform length (n = product of radix[0..npass-1]).
struct FftPlanDev {
  int n;
  int npass;
  int radix[NS3D_MAX_PASSES];
};

// Shared-memory tile accessor: element (col, f) at p[f * ldw + col].
template <typename T>
struct SmemIO {
  cplx<T>* p;
  int ldw;
  NS3D_HD cplx<T> operator()(int col, int f) const { return p[f * ldw + col]; }
  NS3D_HD void operator()(int col, int f, cplx<T> v) const { p[f * ldw + col] = v; }
};

template <typename T, int R, int SIGN, bool COLFAST, class Load, class Store>
NS3D_HD void stockham_pass(int n, int L, int ncol, int tid, int nthr, const cplx<T>* tw,
                           const Load& ld, const Store& st) {
  const int M = n / L;
  const int S = M / R;
  const int ntask = S * L;
  const int total = ntask * ncol;
  for (int w = tid; w < total; w += nthr) {
    int col, task;
    if (COLFAST) {
      col = w % ncol;
      task = w / ncol;
    } else {
      task = w % ntask;
      col = w / ntask;
    }
    const int kap = task % L;
    const int jl = task / L;
    cplx<T> v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = ld(col, (S * q + jl) * L + kap);
    Dft<R, SIGN>::run(v);
    if (S > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) {
        cplx<T> t = tw[jl * k * L];          // w_n^(jl k L) = w_M^(jl k), forward sign
        if (SIGN > 0) t.y = -t.y;
        v[k] = v[k] * t;
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) st(col, jl * L * R + kap + L * k, v[k]);
  }
}

// Radices the generic engine dispatches on (register use is set by the largest).
#define NS3D_FOR_GENERIC_RADICES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(12) X(16)

template <typename T, int SIGN, bool COLFAST, class Load, class Store>
NS3D_HD void dispatch_pass(int r, int n, int L, int ncol, int tid, int nthr, const cplx<T>* tw,
                           const Load& ld, const Store& st) {
  switch (r) {
#define NS3D_CASE(R) \
    case R: stockham_pass<T, R, SIGN, COLFAST>(n, L, ncol, tid, nthr, tw, ld, st); break;
    NS3D_FOR_GENERIC_RADICES(NS3D_CASE)
#undef NS3D_CASE
    default: break;
  }
}

// Buffer the last pass may write into when the result should stay in shared
// memory (the one it does not read): pass 0 writes A, pass i (i >= 1) writes
// B when i is odd, A when even.
template <typename T>
NS3D_HD cplx<T>* fft_free_buffer(int npass, cplx<T>* A, cplx<T>* B) {
  if (npass <= 1) return A;
  return ((npass - 2) % 2 == 0) ? B : A;
}

// Full transform of `ncol` columns of length pl.n.  First pass reads through
// `ld` (mapping FIRST_COLFAST), middle passes ping-pong between A and B, the
// last pass writes through `st` (mapping LAST_COLFAST).  `sync` is a
// block-wide barrier on the device and a no-op on the host.
template <typename T, int SIGN, bool FIRST_COLFAST, bool LAST_COLFAST, class Load, class Store,
          class Sync>
NS3D_HD void fft_tile(const FftPlanDev& pl, int ncol, int tid, int nthr, const cplx<T>* tw,
                      const Load& ld, const Store& st, cplx<T>* A, cplx<T>* B, int ldw,
                      const Sync& sync) {
  const int n = pl.n;
  if (pl.npass == 1) {
    dispatch_pass<T, SIGN, FIRST_COLFAST>(pl.radix[0], n, 1, ncol, tid, nthr, tw, ld, st);
    return;
  }
  SmemIO<T> a{A, ldw}, b{B, ldw};
  int L = 1;
  dispatch_pass<T, SIGN, FIRST_COLFAST>(pl.radix[0], n, L, ncol, tid, nthr, tw, ld, a);
  L *= pl.radix[0];
  sync();
  bool cur_is_a = true;
  for (int p = 1; p < pl.npass - 1; ++p) {
    if (cur_is_a)
      dispatch_pass<T, SIGN, true>(pl.radix[p], n, L, ncol, tid, nthr, tw, a, b);
    else
      dispatch_pass<T, SIGN, true>(pl.radix[p], n, L, ncol, tid, nthr, tw, b, a);
    L *= pl.radix[p];
    cur_is_a = !cur_is_a;
    sync();
  }
  if (cur_is_a)
    dispatch_pass<T, SIGN, LAST_COLFAST>(pl.radix[pl.npass - 1], n, L, ncol, tid, nthr, tw, a, st);
  else
    dispatch_pass<T, SIGN, LAST_COLFAST>(pl.radix[pl.npass - 1], n, L, ncol, tid, nthr, tw, b, st);
}

// Padded-axis index maps.  A retained wavenumber k (|k| <= h - 1, h = N/2) is
// stored at row k mod N of an N-row array and sits at position k mod n of a
// length-n transform.
//   row -> position for an input of `nrow` rows: p < h -> p, p > n - h ->
//   p - n + nrow, otherwise the position is a padding zero (-1).
NS3D_HD int pad_row_of(int p, int n, int h, int nrow) {
  if (p < h) return p;
  if (p > n - h) return p - n + nrow;
  return -1;
}

// Where the positions base .. base + span - 1 of a length-n transform fall for
// a half-width h known at compile time: all below h (kept, low rows), all in
// the zero/dropped band h .. n - h, all above n - h (kept, high rows), or mixed.
enum PadRegion { PAD_LOW = 0, PAD_ZERO = 1, PAD_HIGH = 2, PAD_MIXED = 3 };

NS3D_HDC int pad_region(int base, int span, int n, int h) {
  return (base + span <= h) ? PAD_LOW
         : (base >= h && base + span - 1 <= n - h) ? PAD_ZERO
         : (base > n - h) ? PAD_HIGH
         : PAD_MIXED;
}
