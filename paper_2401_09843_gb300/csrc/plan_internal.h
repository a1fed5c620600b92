// Internal view of a plan for the translation units that extend the C ABI
// (statistics, adjoint); not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include "ns3d.h"
#include "ns3d_geom.h"

namespace ns3d {
struct XFusedMaps;
}

struct LevelView {
  int N = 0, P = 0, B = 0;
  int index = 0;                 // level number in the plan
  const ns3d::Geom* g = nullptr;
  void* U0 = nullptr;
  void* US = nullptr;
  void* W1 = nullptr;
  void* W2 = nullptr;
  void* twP = nullptr;
  Ns3dCtrl* ctrl = nullptr;
  SpecParams sp{};
};

bool find_level(ns3d_plan p, int N, LevelView* out);
bool member_view(ns3d_plan p, int member, LevelView* out, int* index_in_level);
cudaStream_t p_stream(ns3d_plan p);
ns3d_dtype plan_dtype(ns3d_plan p);
const ns3d_params& plan_params(ns3d_plan p);
// synchronises the plan's stream and returns the sticky device status of the level
ns3d_status status_of_level(ns3d_plan p, const LevelView& L);

// Buffers one evaluation of Algorithm 2 + spectral step works on (members
// [0, nm) of the given arrays).
struct StageBufs {
  const ns3d::Geom* g = nullptr;
  SpecParams sp{};
  void* W1 = nullptr;         // workspace A / Cq / Bh
  void* W2 = nullptr;         // workspace Bq / Dq
  const void* tw = nullptr;   // twiddles of length P
  void* u0 = nullptr;         // state at t_n
  void* us = nullptr;         // stage state
  Ns3dCtrl* ctrl = nullptr;   // per member (dt; CFL maximum when wanted)
  // stages 1-3 with the fused x pass: W1 already holds the x-inverse (A) of
  // `in`, and the stage leaves A of `out` in W1 (no separate inverse x)
  bool fused = false;
  const ns3d::XFusedMaps* maps = nullptr;   // TMA descriptors (fused stages)
  const void* lam = nullptr;                 // lambda_k by |k|^2 (fused stages)
  unsigned extra_tx = 0;                     // test hook (ns3d_test_stall_staging)
};

// Optional per-kernel timing: events recorded before each kernel kind.
struct KernelTimer {
  cudaEvent_t ev[7];
};

// Stage 0: out = R(in); stages 1-3: the SSP-RK3 combinations (stage 1 also
// sets each member's dt).  Defined in plan.cu for float and double.
template <typename T>
ns3d_status enqueue_rhs(const StageBufs& b, int stage, int nm, const cplx<T>* in, cplx<T>* out,
                        bool want_umax, cudaStream_t s, KernelTimer* tm = nullptr);

struct PlanDeviceGuard {
  int prev = -1;
  explicit PlanDeviceGuard(ns3d_plan p);
  ~PlanDeviceGuard();
};

struct DevSyncS {
  NS3D_HD void operator()() const {
#if defined(__CUDA_ARCH__)
    __syncthreads();
#endif
  }
};
