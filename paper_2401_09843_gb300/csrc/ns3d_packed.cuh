// Lane types of the packed codelets (codelets_packed.cuh).
//
// A packed codelet runs one small DFT on arrays of real and imaginary parts
// r[], i[] of a lane type V through five operations: padd, psub, pmul (by a
// constant), pfma (constant * a + c) and pneg, with constants pk<V>(c).
//
//   V = float, double   one transform (scalar arithmetic)
//   V = pf2             two independent transforms in lockstep: lane x holds a
//                       value of the first, lane y the same value of the second;
//                       on the GPU each operation is one paired FP32
//                       instruction (add/mul/fma .rn.f32x2 of sm_100 and later),
//                       so both transforms cost the instructions of one.
//
// On the host (the CPU emulator) pf2 runs lane by lane with the same IEEE
// round-to-nearest operations (fmaf for the fused ones), so emulated and GPU
// results agree bit for bit.
#pragma once

#include "ns3d_fft.cuh"

struct alignas(8) pf2 {
  float x, y;
};

NS3D_HD pf2 pf2make(float a, float b) {
  pf2 r;
  r.x = a;
  r.y = b;
  return r;
}

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float2 pf2_v(pf2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ pf2 pf2_of(float2 a) { return pf2make(a.x, a.y); }
#endif

NS3D_HD pf2 padd(pf2 a, pf2 b) {
#if defined(__CUDA_ARCH__)
  return pf2_of(__fadd2_rn(pf2_v(a), pf2_v(b)));
#else
  return pf2make(a.x + b.x, a.y + b.y);
#endif
}

// a - b as the fused b * (-1) + a: the product is exact, so this is the
// correctly rounded difference in one paired instruction
NS3D_HD pf2 psub(pf2 a, pf2 b) {
#if defined(__CUDA_ARCH__)
  return pf2_of(__ffma2_rn(pf2_v(b), make_float2(-1.0f, -1.0f), pf2_v(a)));
#else
  return pf2make(a.x - b.x, a.y - b.y);
#endif
}

NS3D_HD pf2 pmul(pf2 k, pf2 a) {
#if defined(__CUDA_ARCH__)
  return pf2_of(__fmul2_rn(pf2_v(k), pf2_v(a)));
#else
  return pf2make(k.x * a.x, k.y * a.y);
#endif
}

NS3D_HD pf2 pfma(pf2 k, pf2 a, pf2 c) {
#if defined(__CUDA_ARCH__)
  return pf2_of(__ffma2_rn(pf2_v(k), pf2_v(a), pf2_v(c)));
#else
  return pf2make(fmaf(k.x, a.x, c.x), fmaf(k.y, a.y, c.y));
#endif
}

NS3D_HD pf2 pneg(pf2 a) { return pmul(pf2make(-1.0f, -1.0f), a); }

NS3D_HD float padd(float a, float b) { return a + b; }
NS3D_HD float psub(float a, float b) { return a - b; }
NS3D_HD float pmul(float k, float a) { return k * a; }
NS3D_HD float pfma(float k, float a, float c) { return fmaf(k, a, c); }
NS3D_HD float pneg(float a) { return -a; }
NS3D_HD double padd(double a, double b) { return a + b; }
NS3D_HD double psub(double a, double b) { return a - b; }
NS3D_HD double pmul(double k, double a) { return k * a; }
NS3D_HD double pfma(double k, double a, double c) { return fma(k, a, c); }
NS3D_HD double pneg(double a) { return -a; }

template <typename V> NS3D_HD V pk(double c);
template <> NS3D_HD float pk<float>(double c) { return (float)c; }
template <> NS3D_HD double pk<double>(double c) { return c; }
template <> NS3D_HD pf2 pk<pf2>(double c) { return pf2make((float)c, (float)c); }

#include "codelets_packed.cuh"

// A complex value of two lanes: re = (re of lane x, re of lane y), likewise im.
struct pc2 {
  pf2 re, im;
};

// lane-wise complex product with a twiddle w = wr + i wi common to both
// lanes, given as broadcast pairs (wr, wr) and (wi, wi)
NS3D_HD pc2 pc2_twiddle(pc2 a, pf2 wr, pf2 wi) {
  pc2 r;
  r.re = pfma(pneg(wi), a.im, pmul(wr, a.re));
  r.im = pfma(wi, a.re, pmul(wr, a.im));
  return r;
}

// two complex values (lane x, lane y) packed, and back
NS3D_HD pc2 pc2_pack(cplx<float> a, cplx<float> b) {
  pc2 r;
  r.re = pf2make(a.x, b.x);
  r.im = pf2make(a.y, b.y);
  return r;
}
NS3D_HD cplx<float> pc2_lane_x(pc2 a) { return cmake(a.re.x, a.im.x); }
NS3D_HD cplx<float> pc2_lane_y(pc2 a) { return cmake(a.re.y, a.im.y); }
