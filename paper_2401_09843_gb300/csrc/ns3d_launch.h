// Launchers of the solver's kernels.  Each kernel variant lives in its own
// translation unit (col_*.cu, zpass_*.cu, misc_*.cu) so the build compiles
// them in parallel; this header only declares them.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "ns3d_geom.h"
#include "ns3d_zfast.cuh"
#include "ns3d_colfast.cuh"
#include "ns3d_xfused.cuh"
#include "ns3d_colfast3.cuh"
#include "ns3d_zfast3.cuh"

namespace ns3d {

// Column-pass variants: transform direction and the thread mapping of the
// first / last pass (column-fast when the global data is contiguous across
// columns, task-fast when it is contiguous along the transform axis).
enum ColKind {
  COL_INV_CC = 0,   // inverse, contiguous columns in and out (inverse x, inverse y)
  COL_FWD_CC = 3,   // forward, columns in and out (forward y, forward x)
};

template <typename T, int SIGN, bool CF1, bool CFL>
cudaError_t col_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s);
template <typename T, int SIGN, bool CF1, bool CFL>
cudaError_t col_init();

template <typename T, int SIGN, int N1, int N2>
cudaError_t colfast_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s);
template <typename T, int SIGN, int N1, int N2>
cudaError_t colfast_init();

template <typename T, int SIGN, int N1, int N2, int N3>
cudaError_t colfast3_launch(const ColArgs<T>& a, const Launch& L, cudaStream_t s);
template <typename T, int N1, int N2, int N3>
cudaError_t zfast3_launch(const ZArgs<T>& a, int nm, cudaStream_t s);
template <typename T, int N1, int N2, int N3>
cudaError_t long_init();
template <typename T, int N1, int N2, int N3>
cudaError_t zfast3_init();

// A column pass: the register-resident kernel where one exists for (T, n, tile
// width 16) or the three-pass one for long n, the generic tile kernel otherwise.
template <typename T>
cudaError_t launch_col(const ColArgs<T>& a, ColKind kind, const Launch& L, cudaStream_t s) {
  const bool padded_inverse = kind == COL_INV_CC && a.pad_in && !a.trunc_out && a.nrow_in == 2 * a.h;
  const bool truncated_forward = kind == COL_FWD_CC && !a.pad_in && a.trunc_out && a.nrow_out == 2 * a.h;
  // the three-pass kernel indexes rows with 32-bit offsets
  const bool rows32 = (long long)a.pl.n * (a.in_rs > a.out_rs ? a.in_rs : a.out_rs) < (1LL << 31);
  if (sizeof(T) == 4 && 3 * a.h == a.pl.n && rows32 && (padded_inverse || truncated_forward)) {
    const ColArgs<float>& af = *reinterpret_cast<const ColArgs<float>*>(&a);
#define NS3D_CF3_GO(A, B, C)                                                        \
    if (a.pl.n == (A) * (B) * (C))                                                  \
      return kind == COL_INV_CC ? colfast3_launch<float, +1, A, B, C>(af, L, s)    \
                                : colfast3_launch<float, -1, A, B, C>(af, L, s);
    NS3D_FOR_COLFAST3(NS3D_CF3_GO)
#undef NS3D_CF3_GO
  }
  if (sizeof(T) == 8 && 3 * a.h == a.pl.n && rows32 && (padded_inverse || truncated_forward)) {
    const ColArgs<double>& ad = *reinterpret_cast<const ColArgs<double>*>(&a);
#define NS3D_CF3D_GO(A, B, C)                                                        \
    if (a.pl.n == (A) * (B) * (C))                                                   \
      return kind == COL_INV_CC ? colfast3_launch<double, +1, A, B, C>(ad, L, s)    \
                                : colfast3_launch<double, -1, A, B, C>(ad, L, s);
    NS3D_FOR_COLFAST3_F64(NS3D_CF3D_GO)
#undef NS3D_CF3D_GO
  }
  if (sizeof(T) == 4 && a.W == 16 && 3 * a.h == a.pl.n && (padded_inverse || truncated_forward)) {
    const ColArgs<float>& af = *reinterpret_cast<const ColArgs<float>*>(&a);
#define NS3D_CF_GO(A, B)                                                          \
    if (a.pl.n == (A) * (B))                                                      \
      return kind == COL_INV_CC ? colfast_launch<float, +1, A, B>(af, L, s)      \
                                : colfast_launch<float, -1, A, B>(af, L, s);
    NS3D_FOR_COLFAST(NS3D_CF_GO)
#undef NS3D_CF_GO
  }
  switch (kind) {
    case COL_INV_CC: return col_launch<T, +1, true, true>(a, L, s);
    case COL_FWD_CC: return col_launch<T, -1, true, true>(a, L, s);
  }
  return cudaErrorInvalidValue;
}

// TMA descriptors of the fused x pass's inputs (each array of a level viewed
// as FP32 [rows][2 N h], boxes of N/2 rows x 16 complex columns)
struct XFusedMaps {
  CUtensorMap dq, u0, us;
};

// encodes the maps for a level of B members (xfused_maps.cu); false if the
// driver refuses them
bool xfused_make_maps(XFusedMaps* maps, const Geom& g, int B, const void* dq, const void* u0,
                      const void* us);

template <typename T, int N1, int N2>
cudaError_t xfused_launch(const XFusedArgs<T>& a, const XFusedMaps& maps, int nm, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t xfused_prologue_launch(const XFusedArgs<T>& a, int nm, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t xfused_init();

// The fused x pass exists for FP32 at P = N1 N2 with the default padding.
template <typename T>
bool xfused_available(const Geom& g) {
  if (sizeof(T) != 4 || 3 * g.h != g.P || (g.N * g.h) % kXfusedW != 0) return false;
#define NS3D_XF_CASE(A, B) \
  if (g.P == (A) * (B)) return true;
  NS3D_FOR_XFUSED(NS3D_XF_CASE)
#undef NS3D_XF_CASE
  return false;
}

template <typename T>
cudaError_t launch_xfused_prologue(const XFusedArgs<T>& a, const Geom& g, int nm, cudaStream_t s) {
  const XFusedArgs<float>& af = *reinterpret_cast<const XFusedArgs<float>*>(&a);
#define NS3D_XFP_GO(A, B) \
  if (g.P == (A) * (B)) return xfused_prologue_launch<float, A, B>(af, nm, s);
  NS3D_FOR_XFUSED(NS3D_XFP_GO)
#undef NS3D_XFP_GO
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_xfused(const XFusedArgs<T>& a, const XFusedMaps& maps, const Geom& g, int nm,
                          cudaStream_t s) {
  const XFusedArgs<float>& af = *reinterpret_cast<const XFusedArgs<float>*>(&a);
#define NS3D_XF_GO(A, B) \
  if (g.P == (A) * (B)) return xfused_launch<float, A, B>(af, maps, nm, s);
  NS3D_FOR_XFUSED(NS3D_XF_GO)
#undef NS3D_XF_GO
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_zfused(const ZArgs<T>& a, const Launch& L, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t zfast_launch(const ZArgs<T>& a, int nm, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t zfast_init();
template <typename T, int N1, int N2>
cudaError_t zrot_launch(const ZArgs<T>& a, int nm, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t zrot_init();
template <typename T, int N1, int N2>
cudaError_t zadjf_launch(const ZArgs<T>& a, int nm, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t zadjf_init();
template <typename T, int N1, int N2>
cudaError_t zadv_launch(const ZArgs<T>& a, int nm, cudaStream_t s);
template <typename T, int N1, int N2>
cudaError_t zadv_init();


template <typename T>
bool zfast3_available(int P) {
#define NS3D_ZF3_CASE(A, B, C) \
  if (P == (A) * (B) * (C)) return true;
  if (sizeof(T) == 4) {
    NS3D_FOR_ZFAST3(NS3D_ZF3_CASE)
  } else {
    NS3D_FOR_ZFAST3_F64(NS3D_ZF3_CASE)
  }
#undef NS3D_ZF3_CASE
  return false;
}

template <typename T>
bool zfast_available(int P) {
  if (sizeof(T) != 4) return false;
#define NS3D_ZF_CASE(A, B) \
  if (P == (A) * (B)) return true;
  NS3D_FOR_ZFAST(NS3D_ZF_CASE)
#undef NS3D_ZF_CASE
  return false;
}

// the rotational form's register-resident z pass exists for this level
inline bool zrot_available(const Geom& g) {
  return g.form == 2 && g.esz == 8 && 3 * g.h == g.P && zfast_available<float>(g.P);
}

// the advective form's register-resident z pass exists for this level
inline bool zadv_available(const Geom& g) {
  return g.form == 1 && g.esz == 8 && 3 * g.h == g.P && zfast_available<float>(g.P);
}

// a form-1/2 level whose z pass is register-resident (no tile to tune)
inline bool zform_register(const Geom& g) { return zrot_available(g) || zadv_available(g); }



// The fused z pass of a level: the register-resident kernel where one exists
// for (T, P), the generic tile kernel otherwise.
template <typename T>
cudaError_t launch_zpass(const ZArgs<T>& a, const Geom& g, int nm, cudaStream_t s);
template <typename T>
cudaError_t zfused_init();
template <typename T>
cudaError_t launch_spectral(const SpecArgs<T>& a, cudaStream_t s);
// nonlinear forms 1 and 2: the form's spectral fields, and the z pass with products
template <typename T>
cudaError_t launch_form_prep(const cplx<T>* u, cplx<T>* F, int N, T kscale, int form, long long mu,
                             long long mf, int nm, cudaStream_t s);
template <typename T>
cudaError_t launch_zform(const ZArgs<T>& a, int form, const Launch& L, cudaStream_t s);
template <typename T>
cudaError_t zform_init();

// z pass of a form-1/2 level: the rotational or advective register kernel
// where it exists, else the tuned zform tile kernel
template <typename T>
cudaError_t launch_zform_level(const ZArgs<T>& a, const Geom& g, int nm, cudaStream_t s) {
  if (sizeof(T) == 4 && zrot_available(g)) {
    const ZArgs<float>& af = *reinterpret_cast<const ZArgs<float>*>(&a);
#define NS3D_ZR_GO(A, B) \
    if (g.P == (A) * (B)) return zrot_launch<float, A, B>(af, nm, s);
    NS3D_FOR_ZFAST(NS3D_ZR_GO)
#undef NS3D_ZR_GO
  }
  if (sizeof(T) == 4 && zadv_available(g)) {
    const ZArgs<float>& af = *reinterpret_cast<const ZArgs<float>*>(&a);
#define NS3D_ZA_GO(A, B) \
    if (g.P == (A) * (B)) return zadv_launch<float, A, B>(af, nm, s);
    NS3D_FOR_ZFAST(NS3D_ZA_GO)
#undef NS3D_ZA_GO
  }
  return launch_zform<T>(a, g.form, Launch{cdiv(g.P, g.Wzf), g.P, nm, g.nthr_zf, g.smem_zf}, s);
}
// per-member time step of the step starting now (before the stage-1 spectral kernel)
cudaError_t launch_step_dt(Ns3dCtrl* c, int n, const SpecParams& sp, cudaStream_t s);
template <typename T>
cudaError_t launch_d1_to_compact(const cplx<T>* d1, cplx<T>* u, int N, cudaStream_t s);
template <typename T>
cudaError_t launch_compact_to_d1(const cplx<T>* u, cplx<T>* d1, int N, cudaStream_t s);

template <typename T>
cudaError_t kernels_init() {
  cudaError_t e[4] = {col_init<T, +1, true, true>(), col_init<T, -1, true, true>(),
                      zfused_init<T>(), zform_init<T>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  if (sizeof(T) == 8) {
#define NS3D_Z64_INIT(A, B, C)                              \
    {                                                       \
      cudaError_t r = zfast3_init<double, A, B, C>();       \
      if (r != cudaSuccess) return r;                       \
    }
    NS3D_FOR_ZFAST3_F64(NS3D_Z64_INIT)
#undef NS3D_Z64_INIT
#define NS3D_LONG64_INIT(A, B, C)                           \
    {                                                       \
      cudaError_t r = long_init<double, A, B, C>();         \
      if (r != cudaSuccess) return r;                       \
    }
    NS3D_FOR_COLFAST3_F64(NS3D_LONG64_INIT)
#undef NS3D_LONG64_INIT
  }
  if (sizeof(T) == 4) {
#define NS3D_ZF_INIT(A, B)                                  \
    {                                                       \
      cudaError_t r = zfast_init<float, A, B>();            \
      if (r == cudaSuccess) r = zrot_init<float, A, B>();   \
      if (r == cudaSuccess) r = zadjf_init<float, A, B>();  \
      if (r == cudaSuccess) r = zadv_init<float, A, B>();   \
      if (r != cudaSuccess) return r;                       \
    }
    NS3D_FOR_ZFAST(NS3D_ZF_INIT)
#undef NS3D_ZF_INIT
#define NS3D_LONG_INIT(A, B, C)                             \
    {                                                       \
      cudaError_t r = long_init<float, A, B, C>();          \
      if (r != cudaSuccess) return r;                       \
    }
    NS3D_FOR_COLFAST3(NS3D_LONG_INIT)
#undef NS3D_LONG_INIT
#define NS3D_Z3_INIT(A, B, C)                               \
    {                                                       \
      cudaError_t r = zfast3_init<float, A, B, C>();        \
      if (r != cudaSuccess) return r;                       \
    }
    NS3D_FOR_ZFAST3(NS3D_Z3_INIT)
#undef NS3D_Z3_INIT
#define NS3D_XF_INIT(A, B)                                  \
    {                                                       \
      cudaError_t r = xfused_init<float, A, B>();           \
      if (r != cudaSuccess) return r;                       \
    }
    NS3D_FOR_XFUSED(NS3D_XF_INIT)
#undef NS3D_XF_INIT
#define NS3D_CF_INIT(A, B)                                                         \
    {                                                                              \
      cudaError_t r1 = colfast_init<float, +1, A, B>();                            \
      cudaError_t r2 = colfast_init<float, -1, A, B>();                            \
      if (r1 != cudaSuccess) return r1;                                            \
      if (r2 != cudaSuccess) return r2;                                            \
    }
    NS3D_FOR_COLFAST(NS3D_CF_INIT)
#undef NS3D_CF_INIT
  }
  return cudaSuccess;
}

cudaError_t launch_ctrl_reset(Ns3dCtrl* c, int n, cudaStream_t s);
cudaError_t launch_ctrl_set_tend(Ns3dCtrl* c, int n, double t_end, cudaStream_t s);
cudaError_t launch_ctrl_set_clock(Ns3dCtrl* c, double t, int nsteps, cudaStream_t s);

}  // namespace ns3d
