// Double-single arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, a 48-bit significand (unit roundoff about
// 2^-48 = 3.6e-15) in FP32's exponent range.
//
// GB300 runs FP32 at 64 times its FP64 rate, and the FP64 transforms of the
// solver are bound by that FP64 rate, so the long-line transforms of FP64
// plans compute in this type: the data stay IEEE binary64 in memory and are
// split exactly into (hi, lo) on load (hi = fl32(d), lo = fl32(d - hi)) and
// joined on store (hi + lo in binary64).  The operations follow the
// error-free transformations of Knuth (TwoSum: s = fl(a + b) and its exact
// error), Dekker's fast renormalisation, and the FMA form of TwoProduct
// (p = fl(a b), e = fma(a, b, -p) exactly): the sum adds the two high parts
// exactly, then the low parts, and renormalises ("sloppy" addition, an
// absolute error of a few units of 2^-48 times |a| + |b|, which is the bound
// an FFT's error analysis uses); the product is accurate to a few units of
// 2^-48 relative.
//
// On the GPU every FP32 operation is an explicitly rounded intrinsic, so the
// compiler never fuses a product into a later sum (which would break the
// error-free steps); on the host (the CPU emulator) plain single-precision
// operations and fmaf give the same roundings, so both agree bit for bit.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define NS3D_DF_HD __host__ __device__ __forceinline__
#else
#define NS3D_DF_HD inline
#endif

namespace dfops {
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float add(float a, float b) { return a + b; }
inline float sub(float a, float b) { return a - b; }
inline float mul(float a, float b) { return a * b; }
inline float fma(float a, float b, float c) { return fmaf(a, b, c); }
#endif
}  // namespace dfops

struct df64 {
  float hi, lo;
  df64() = default;
  NS3D_DF_HD df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  NS3D_DF_HD df64(float f) : hi(f), lo(0.0f) {}
  NS3D_DF_HD df64(int i) : hi((float)i), lo(0.0f) {}
  NS3D_DF_HD static df64 raw(float h, float l) {
    df64 r;
    r.hi = h;
    r.lo = l;
    return r;
  }
  NS3D_DF_HD explicit operator double() const { return (double)hi + (double)lo; }
};

// (h, l) = Dekker's renormalisation of s + e for |s| >= |e|
NS3D_DF_HD df64 df_fast_two_sum(float s, float e) {
  const float h = dfops::add(s, e);
  const float l = dfops::sub(e, dfops::sub(h, s));
  return df64::raw(h, l);
}

NS3D_DF_HD df64 operator+(df64 a, df64 b) {
  const float s = dfops::add(a.hi, b.hi);
  const float bb = dfops::sub(s, a.hi);
  float e = dfops::add(dfops::sub(a.hi, dfops::sub(s, bb)), dfops::sub(b.hi, bb));   // exact error
  e = dfops::add(e, dfops::add(a.lo, b.lo));
  return df_fast_two_sum(s, e);
}

NS3D_DF_HD df64 operator-(df64 a) { return df64::raw(-a.hi, -a.lo); }
NS3D_DF_HD df64 operator-(df64 a, df64 b) { return a + (-b); }

NS3D_DF_HD df64 operator*(df64 a, df64 b) {
  const float p = dfops::mul(a.hi, b.hi);
  float e = dfops::fma(a.hi, b.hi, -p);                                 // exact error of p
  e = dfops::fma(a.hi, b.lo, e);
  e = dfops::fma(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

NS3D_DF_HD bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
NS3D_DF_HD bool operator>(df64 a, df64 b) { return b < a; }
NS3D_DF_HD bool operator<=(df64 a, df64 b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
NS3D_DF_HD bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }

NS3D_DF_HD df64 xabs(df64 a) { return a.hi < 0.0f ? -a : a; }
// maximum that ignores a NaN operand (as fmax)
NS3D_DF_HD df64 xmax(df64 a, df64 b) {
  if (!(a.hi == a.hi)) return b;
  if (!(b.hi == b.hi)) return a;
  return a < b ? b : a;
}

#include "ns3d_fft.cuh"

// Arithmetic type of the long-line (three-pass) register kernels for a
// storage type T: FP32 computes in FP32, FP64 in double-single.
template <typename T> struct LongArith { using type = T; };
template <> struct LongArith<double> { using type = df64; };
template <typename T> using LongC = typename LongArith<T>::type;

// complex value converted between storage and arithmetic types (exact from
// binary64 to double-single; hi + lo rounded once back to binary64)
template <typename C, typename T>
NS3D_DF_HD cplx<C> ccvt(cplx<T> v) {
  return cmake((C)v.x, (C)v.y);
}
