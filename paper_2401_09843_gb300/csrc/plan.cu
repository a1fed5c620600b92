// C ABI of the solver (include/ns3d.h): plans, workspaces, the captured
// step graph, state transfer and the right-hand-side evaluation.
//
// A plan groups its members by resolution into levels.  Each level owns
//   U0   state u_n              [B][3][N][N][N/2]
//   US   stage state u1 / u2    [B][3][N][N][N/2]
//   W1   A  / Cq / Bh           (aliased workspaces, Workspaces of section 3.4:
//   W2   Bq / Dq                 each is dead before the next pass reuses it)
// and one RK3 stage is the pass sequence
//   inverse x (pad) -> inverse y (pad) -> z: c2r, products, r2c (truncate)
//   -> forward y (truncate) -> forward x (truncate) -> spectral step + combine,
// i.e. Algorithm 2 with the padding fused into the transforms (Algorithm 3).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ns3d.h"
#include "ns3d_launch.h"
#include "plan_internal.h"

using namespace ns3d;

namespace {

struct Level {
  int N = 0, P = 0, B = 0;
  Geom g;
  SpecParams sp{};
  std::vector<int> members;
  void* U0 = nullptr;
  void* US = nullptr;
  void* W1 = nullptr;
  void* W2 = nullptr;
  void* twP = nullptr;
  Ns3dCtrl* ctrl = nullptr;
  bool fused = false;     // the step uses the fused x pass (FP32 register sizes)
  bool a_valid = false;   // W1 holds the x-inverse of U0 (set by the last step)
  XFusedMaps maps{};      // TMA descriptors of W2 (Dq), U0, US for the fused x pass
  void* lamT = nullptr;   // lambda_k by |k|^2 in the arithmetic type
  unsigned extra_tx = 0;  // test hook: bytes the first staged tile never delivers
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// NVTX range over one C-ABI call (visible in Nsight Systems timelines)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

struct ns3d_plan_s {
  int device = 0;
  ns3d_dtype dtype = NS3D_F32;
  int esz = 8;
  ns3d_params prm{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<Level> levels;
  std::vector<std::pair<int, int>> loc;  // member -> (level, index in level)
  std::vector<void*> allocs;
  size_t bytes = 0;
  void* staging = nullptr;               // device buffer of one member in D1 layout
  size_t staging_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double t_end = 0.0;
  int launches_per_step = 0;
};

#define NS3D_CK(x)                            \
  do {                                        \
    if ((x) != cudaSuccess) return NS3D_ERR_CUDA; \
  } while (0)

extern "C" void ns3d_params_default(ns3d_params* p) {
  if (!p) return;
  p->L = 6.283185307179586476925286766559;
  p->nu = 0.0;
  p->s = 1.5;
  p->theta = 0.5;
  p->eps0 = 1.0;
  p->mN_coef = 1.0;
  p->q_form = 0;
  p->n_pad = 0;
  p->nonlinear_form = 0;
  p->cfl = 0.5;
  p->dt_fixed = 0.0;
}

extern "C" const char* ns3d_status_string(ns3d_status s) {
  switch (s) {
    case NS3D_OK: return "ok";
    case NS3D_ERR_INVALID_ARG: return "invalid argument";
    case NS3D_ERR_OUT_OF_MEMORY: return "out of memory";
    case NS3D_ERR_CUDA: return "CUDA error";
    case NS3D_ERR_NONFINITE: return "non-finite velocity";
    case NS3D_ERR_UNSTABLE_DT: return "time step above the RK3 stability limit";
    case NS3D_ERR_TIMEOUT: return "device wait timed out";
    case NS3D_ERR_NOT_SUPPORTED: return "not supported";
  }
  return "unknown status";
}

namespace {

ns3d_status dev_alloc(ns3d_plan p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return NS3D_OK;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return NS3D_ERR_OUT_OF_MEMORY;
  }
  p->allocs.push_back(*ptr);
  p->bytes += bytes;
  return NS3D_OK;
}

void free_all(ns3d_plan p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
  if (p->cap) cudaStreamDestroy(p->cap);
  p->cap = nullptr;
}

template <typename T>
ns3d_status upload_twiddles(Level& L, cudaStream_t s) {
  std::vector<cplx<T>> tw = make_twiddles<T>(L.P);
  NS3D_CK(cudaMemcpyAsync(L.twP, tw.data(), tw.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice, s));
  NS3D_CK(cudaStreamSynchronize(s));
  return NS3D_OK;
}

// lambda_k by integer |k|^2 over the retained band (0 .. 3 (h - 1)^2),
// evaluated in double and rounded once to the arithmetic type
template <typename T>
ns3d_status upload_lambda(Level& L, cudaStream_t s) {
  const int hm = L.g.h - 1;
  const SpecT<double> sp = spec_t<double>(L.sp);
  std::vector<T> lam(3 * hm * hm + 1);
  for (size_t k2 = 0; k2 < lam.size(); ++k2) lam[k2] = T(lambda_k<double>((int)k2, sp));
  NS3D_CK(cudaMemcpyAsync(L.lamT, lam.data(), lam.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  NS3D_CK(cudaStreamSynchronize(s));
  return NS3D_OK;
}

size_t lambda_entries(const Geom& g) { return 3 * (size_t)(g.h - 1) * (g.h - 1) + 1; }

// One evaluation of Algorithm 2 plus the spectral step for members
// [m0, m0 + nm) of a level.  `in` is the field R is evaluated at; stage 0
// writes R to `out`, stages 1-3 the SSP-RK3 combinations.
// kernel kinds of one stage, for CUDA events and NVTX ranges (eager timing)
const char* const kKindNames[6] = {"inverse x", "inverse y", "z pass", "forward y", "forward x",
                                   "spectral / fused x"};

#define NS3D_MARK(i)                                      \
  if (tm) {                                               \
    NS3D_CK(cudaEventRecord(tm->ev[i], s));               \
    if ((i) > 0) nvtxRangePop();                          \
    if ((i) < 6) nvtxRangePushA(kKindNames[(i) < 6 ? (i) : 0]); \
  }

StageBufs level_bufs(Level& L, int m0) {
  StageBufs b;
  b.g = &L.g;
  b.sp = L.sp;
  b.W1 = L.W1;
  b.W2 = L.W2;
  b.tw = L.twP;
  b.u0 = static_cast<unsigned char*>(L.U0) + (size_t)m0 * L.g.nU * L.g.esz;
  b.us = static_cast<unsigned char*>(L.US) + (size_t)m0 * L.g.nU * L.g.esz;
  b.ctrl = L.ctrl + m0;
  b.fused = false;
  b.lam = L.lamT;
  return b;
}

template <typename T>
ns3d_status enqueue_stage(Level& L, int stage, int m0, int nm, const cplx<T>* in, cplx<T>* out,
                          bool want_umax, cudaStream_t s, KernelTimer* tm = nullptr) {
  StageBufs b = level_bufs(L, m0);
  b.fused = L.fused && stage >= 1 && m0 == 0 && nm == L.B;
  b.maps = &L.maps;
  b.extra_tx = L.extra_tx;
  return enqueue_rhs<T>(b, stage, nm, in, out, want_umax, s, tm);
}

// x-inverse of every member's state into W1 (needed before the first fused
// stage after the state or W1 changed outside a step)
// (with the fused pass's own inverse phases, so that a state set from a
// checkpoint continues bit for bit as if the run had not stopped)
template <typename T>
ns3d_status enqueue_prologue(Level& L, cudaStream_t s) {
  XFusedArgs<T> x{};
  x.u0 = static_cast<const cplx<T>*>(L.U0);
  x.ax = static_cast<cplx<T>*>(L.W1);
  x.tw = static_cast<const cplx<T>*>(L.twP);
  x.N = L.g.N;
  x.h = L.g.h;
  x.m3 = L.g.nU;
  x.mA = L.g.nA;
  NS3D_CK(launch_xfused_prologue<T>(x, L.g, L.B, s));
  L.a_valid = true;
  return NS3D_OK;
}

ns3d_status ensure_prologue(ns3d_plan p) {
  for (Level& L : p->levels) {
    if (!L.fused || L.a_valid) continue;
    ns3d_status st = p->dtype == NS3D_F32 ? enqueue_prologue<float>(L, p->stream)
                                          : enqueue_prologue<double>(L, p->stream);
    if (st != NS3D_OK) return st;
  }
  return NS3D_OK;
}

}  // namespace

namespace {

// enqueue_rhs for the advective (1) and rotational (2) forms: the form's nf
// spectral fields, their inverse x and y passes, the z pass that forms the
// three products, forward y and x of the products and the spectral step with
// b taken as it is (no kappa contraction).
template <typename T>
ns3d_status enqueue_rhs_form(const StageBufs& b, int stage, int nm, const cplx<T>* in,
                             cplx<T>* out, bool want_umax, cudaStream_t s, KernelTimer* tm) {
  const Geom& g = *b.g;
  const long long N = g.N, P = g.P, h = g.h;
  const int nf = form_fields(g.form);
  cplx<T>* W1 = static_cast<cplx<T>*>(b.W1);
  cplx<T>* W2 = static_cast<cplx<T>*>(b.W2);
  const cplx<T>* tw = static_cast<const cplx<T>*>(b.tw);
  NS3D_MARK(0);
  NS3D_CK(launch_form_prep<T>(in, W1, g.N, T(b.sp.kscale), g.form, g.nU, nf * N * N * h, nm, s));
  Launch lx = launch_inv_x(g, nm);
  lx.gz = nm * nf;
  NS3D_CK(launch_col<T>(args_inv_x<T>(g, W1, W2, tw), COL_INV_CC, lx, s));
  NS3D_MARK(1);
  Launch ly = launch_inv_y(g, nm);
  ly.gz = nm * nf;
  NS3D_CK(launch_col<T>(args_inv_y<T>(g, W2, W1, tw), COL_INV_CC, ly, s));
  NS3D_MARK(2);
  ZArgs<T> az = args_z<T>(g, W1, W2, tw, want_umax ? b.ctrl : nullptr);
  az.W = g.Wzf;
  az.ldw = g.ldwzf;
  az.in_bs = nf * P * P * h;
  az.out_bs = 3 * P * P * h;
  NS3D_CK(launch_zform_level<T>(az, g, nm, s));
  NS3D_MARK(3);
  Launch lfy = launch_fwd_y(g, nm);
  lfy.gz = nm * 3;
  NS3D_CK(launch_col<T>(args_fwd_y<T>(g, W2, W1, tw), COL_FWD_CC, lfy, s));
  NS3D_MARK(4);
  Launch lfx = launch_fwd_x(g, nm);
  lfx.gz = nm * 3;
  NS3D_CK(launch_col<T>(args_fwd_x<T>(g, W1, W2, tw), COL_FWD_CC, lfx, s));
  NS3D_MARK(5);
  SpecArgs<T> a{};
  a.bh = W2;
  a.u0 = (stage == 0) ? in : static_cast<cplx<T>*>(b.u0);
  a.us = static_cast<cplx<T>*>(b.us);
  a.out = out;
  a.N = g.N;
  a.h = g.h;
  a.nmem = nm;
  a.stage = stage;
  a.m6 = 3 * N * N * h;
  a.m3 = g.nU;
  a.sp = spec_t<T>(b.sp);
  a.ctrl = b.ctrl;
  a.lam = static_cast<const T*>(b.lam);
  a.form = g.form;
  if (stage == 1) NS3D_CK(launch_step_dt(b.ctrl, nm, b.sp, s));
  NS3D_CK(launch_spectral<T>(a, s));
  NS3D_MARK(6);
  return NS3D_OK;
}

}  // namespace

// One evaluation of Algorithm 2 plus the spectral step for members [0, nm)
// of the buffers.  `in` is the field R is evaluated at; stage 0 writes R to
// `out`, stages 1-3 the SSP-RK3 combinations.
template <typename T>
ns3d_status enqueue_rhs(const StageBufs& b, int stage, int nm, const cplx<T>* in, cplx<T>* out,
                        bool want_umax, cudaStream_t s, KernelTimer* tm) {
  const Geom& g = *b.g;
  if (g.form != 0) return enqueue_rhs_form<T>(b, stage, nm, in, out, want_umax, s, tm);
  cplx<T>* W1 = static_cast<cplx<T>*>(b.W1);
  cplx<T>* W2 = static_cast<cplx<T>*>(b.W2);
  const cplx<T>* tw = static_cast<const cplx<T>*>(b.tw);
  cplx<T>* U0 = static_cast<cplx<T>*>(b.u0);
  cplx<T>* US = static_cast<cplx<T>*>(b.us);
  NS3D_MARK(0);
  if (!b.fused)
    NS3D_CK(launch_col<T>(args_inv_x<T>(g, in, W1, tw), COL_INV_CC, launch_inv_x(g, nm), s));
  NS3D_MARK(1);
  NS3D_CK(launch_col<T>(args_inv_y<T>(g, W1, W2, tw), COL_INV_CC, launch_inv_y(g, nm), s));
  NS3D_MARK(2);
  NS3D_CK(launch_zpass<T>(args_z<T>(g, W2, W1, tw, want_umax ? b.ctrl : nullptr), g, nm, s));
  NS3D_MARK(3);
  NS3D_CK(launch_col<T>(args_fwd_y<T>(g, W1, W2, tw), COL_FWD_CC, launch_fwd_y(g, nm), s));
  NS3D_MARK(4);
  if (b.fused) {
    // forward x + spectral step + RK3 combine + inverse x of the new state
    XFusedArgs<T> x{};
    x.dq = W2;
    x.u0 = U0;
    x.us = US;
    x.out = out;
    x.ax = W1;
    x.tw = tw;
    x.lam = static_cast<const T*>(b.lam);
    x.extra_tx = b.extra_tx;
    x.N = g.N;
    x.h = g.h;
    x.stage = stage;
    x.m6 = g.nDq;
    x.m3 = g.nU;
    x.mA = g.nA;
    x.sp = spec_t<T>(b.sp);
    x.ctrl = b.ctrl;
    NS3D_MARK(5);
    if (stage == 1) NS3D_CK(launch_step_dt(b.ctrl, nm, b.sp, s));
    NS3D_CK(launch_xfused<T>(x, *b.maps, g, nm, s));
    NS3D_MARK(6);
    return NS3D_OK;
  }
  NS3D_CK(launch_col<T>(args_fwd_x<T>(g, W2, W1, tw), COL_FWD_CC, launch_fwd_x(g, nm), s));
  NS3D_MARK(5);
  SpecArgs<T> a{};
  a.bh = W1;
  a.u0 = (stage == 0) ? in : U0;
  a.us = US;
  a.out = out;
  a.N = g.N;
  a.h = g.h;
  a.nmem = nm;
  a.stage = stage;
  a.m6 = g.nBh;
  a.m3 = g.nU;
  a.sp = spec_t<T>(b.sp);
  a.ctrl = b.ctrl;
  a.lam = static_cast<const T*>(b.lam);
  if (stage == 1) NS3D_CK(launch_step_dt(b.ctrl, nm, b.sp, s));
  NS3D_CK(launch_spectral<T>(a, s));
  NS3D_MARK(6);
  return NS3D_OK;
}

template ns3d_status enqueue_rhs<float>(const StageBufs&, int, int, const cplx<float>*, cplx<float>*,
                                        bool, cudaStream_t, KernelTimer*);
template ns3d_status enqueue_rhs<double>(const StageBufs&, int, int, const cplx<double>*,
                                         cplx<double>*, bool, cudaStream_t, KernelTimer*);

namespace {

template <typename T>
ns3d_status enqueue_step(ns3d_plan p, cudaStream_t s) {
  for (Level& L : p->levels) {
    cplx<T>* U0 = static_cast<cplx<T>*>(L.U0);
    cplx<T>* US = static_cast<cplx<T>*>(L.US);
    ns3d_status st;
    if ((st = enqueue_stage<T>(L, 1, 0, L.B, U0, US, p->prm.dt_fixed <= 0, s)) != NS3D_OK) return st;
    if ((st = enqueue_stage<T>(L, 2, 0, L.B, US, US, false, s)) != NS3D_OK) return st;
    if ((st = enqueue_stage<T>(L, 3, 0, L.B, US, U0, false, s)) != NS3D_OK) return st;
  }
  return NS3D_OK;
}

ns3d_status build_graph(ns3d_plan p) {
  if (p->exec) return NS3D_OK;
  NS3D_CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
  ns3d_status st = p->dtype == NS3D_F32 ? enqueue_step<float>(p, p->cap) : enqueue_step<double>(p, p->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(p->cap, &g);
  if (st != NS3D_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return NS3D_ERR_CUDA;
  p->graph = g;
  if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
    p->exec = nullptr;
    return NS3D_ERR_CUDA;
  }
  return NS3D_OK;
}

ns3d_status member_lookup(ns3d_plan p, int member, Level** L, int* idx) {
  if (!p || member < 0 || member >= (int)p->loc.size()) return NS3D_ERR_INVALID_ARG;
  *L = &p->levels[p->loc[member].first];
  *idx = p->loc[member].second;
  return NS3D_OK;
}

size_t d1_bytes(int N, int esz) { return (size_t)3 * N * N * (N / 2 + 1) * esz; }

// D1 (device or host) -> compact member slot
template <typename T>
ns3d_status put_d1(ns3d_plan p, Level& L, const void* src, int on_device, cplx<T>* dst) {
  const size_t nb = d1_bytes(L.N, p->esz);
  const void* dsrc = src;
  if (!on_device) {
    NS3D_CK(cudaMemcpyAsync(p->staging, src, nb, cudaMemcpyHostToDevice, p->stream));
    dsrc = p->staging;
  }
  NS3D_CK(launch_d1_to_compact<T>(static_cast<const cplx<T>*>(dsrc), dst, L.N, p->stream));
  return NS3D_OK;
}

template <typename T>
ns3d_status get_d1(ns3d_plan p, Level& L, const cplx<T>* src, void* dst, int on_device) {
  const size_t nb = d1_bytes(L.N, p->esz);
  void* ddst = on_device ? dst : p->staging;
  NS3D_CK(launch_compact_to_d1<T>(src, static_cast<cplx<T>*>(ddst), L.N, p->stream));
  if (!on_device) NS3D_CK(cudaMemcpyAsync(dst, p->staging, nb, cudaMemcpyDeviceToHost, p->stream));
  return NS3D_OK;
}

ns3d_status status_of_flags(int flags) {
  // a timed-out stage leaves its output undefined: report the cause first
  if (flags & NS3D_FLAG_TIMEOUT) return NS3D_ERR_TIMEOUT;
  if (flags & NS3D_FLAG_NONFINITE) return NS3D_ERR_NONFINITE;
  if (flags & NS3D_FLAG_UNSTABLE) return NS3D_ERR_UNSTABLE_DT;
  return NS3D_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------- autotune
// The padded size (section 3.1): the smallest 2^a 3^b 5^c 7^d >= 3N/2 unless
// a benchmark of a few larger candidates says otherwise.  Where the register
// kernels exist (FP32 at P = 3N/2) the smallest size is taken without one.

bool register_kernels_at(int N, int P, ns3d_dtype dtype) {
  if (2 * P != 3 * N) return false;
  if (dtype == NS3D_F64) return zfast3_available<double>(P);   // double-single three-pass kernels
  return zfast_available<float>(P) || zfast3_available<float>(P);
}

std::vector<int> pad_candidates(int N) {
  std::vector<int> c;
  const int P0 = default_padded_size(N);
  for (int P = P0; P <= P0 + P0 / 8 && c.size() < 4; ++P)
    if (is_7_smooth(P)) c.push_back(P);
  return c;
}

std::mutex g_tune_mu;
std::map<std::tuple<std::string, int, int>, int> g_tune;   // (device, N, dtype) -> P
bool g_tune_loaded = false;

// optional cache file (environment NS3D_AUTOTUNE_CACHE): lines "device<TAB>N dtype P"
void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("NS3D_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    char* tab = std::strchr(line, '\t');
    if (!tab) continue;
    int N = 0, dt = 0, P = 0;
    if (std::sscanf(tab + 1, "%d %d %d", &N, &dt, &P) == 3 && 2 * P >= 3 * N)
      g_tune[std::make_tuple(std::string(line, tab), N, dt)] = P;
  }
  std::fclose(f);
}

void tune_cache_store(const std::string& dev, int N, int dt, int P) {
  const char* path = std::getenv("NS3D_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s\t%d %d %d\n", dev.c_str(), N, dt, P);
  std::fclose(f);
}

// milliseconds of one right-hand side at (N, P) through the public entry
// points, best of three after a warm-up; negative if the size cannot be run
double time_rhs(int N, int P, ns3d_dtype dtype, ns3d_params prm, cudaStream_t s) {
  prm.n_pad = P;
  ns3d_plan tp = nullptr;
  if (ns3d_plan_create(&tp, &N, 1, dtype, &prm, s, 0) != NS3D_OK) return -1.0;
  const size_t bytes = d1_bytes(N, dtype == NS3D_F32 ? 8 : 16);
  void* in = nullptr;
  void* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = -1.0;
  if (cudaMalloc(&in, bytes) == cudaSuccess && cudaMalloc(&out, bytes) == cudaSuccess &&
      cudaMemsetAsync(in, 0, bytes, s) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess && ns3d_eval_rhs(tp, 0, in, out, 1) == NS3D_OK) {
    for (int r = 0; r < 3; ++r) {
      float ms = 0.f;
      if (cudaEventRecord(e0, s) != cudaSuccess || ns3d_eval_rhs(tp, 0, in, out, 1) != NS3D_OK ||
          cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        best = -1.0;
        break;
      }
      if (best < 0 || ms < best) best = ms;
    }
  }
  cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (in) cudaFree(in);
  if (out) cudaFree(out);
  ns3d_plan_destroy(tp);
  return best;
}

// (device, N, P, dtype, form) -> index into form_tile_candidates
std::map<std::tuple<std::string, int, int, int, int>, int> g_form_tile;

// The zform tile of a form-1/2 level: each candidate shape timed on the first
// x planes (at most 96) of member 0 in the level's own workspaces (zeroed
// fields; one warm-up and two timed launches), the fastest kept and cached per
// device.  The shape does not change the computed values.
template <typename T>
ns3d_status tune_form_tile(Level& L, ns3d_dtype dtype, cudaStream_t s) {
  Geom& g = L.g;
  const std::vector<FormTile> cand = form_tile_candidates(g);
  if (cand.empty()) return NS3D_ERR_NOT_SUPPORTED;
  int dev = 0;
  cudaDeviceProp pr{};
  std::string name = "unknown";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&pr, dev) == cudaSuccess)
    name = pr.name;
  const auto key = std::make_tuple(name, g.N, g.P, (int)dtype, g.form);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_form_tile.find(key);
    if (it != g_form_tile.end()) {
      set_form_tile(&g, cand[it->second]);
      return NS3D_OK;
    }
  }
  const long long P = g.P, h = g.h;
  const int nf = form_fields(g.form);
  NS3D_CK(cudaMemsetAsync(L.W1, 0, (size_t)nf * P * P * h * sizeof(cplx<T>), s));
  ZArgs<T> az = args_z<T>(g, static_cast<const cplx<T>*>(L.W1), static_cast<cplx<T>*>(L.W2),
                          static_cast<const cplx<T>*>(L.twP), nullptr);
  az.in_bs = nf * P * P * h;
  az.out_bs = 3 * P * P * h;
  const int gy = (int)std::min<long long>(P, 96);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return NS3D_ERR_CUDA;
  }
  int best = -1;
  float best_ms = 0.f;
  for (size_t c = 0; c < cand.size(); ++c) {
    az.W = cand[c].W;
    az.ldw = cand[c].W + 1;
    const Launch lz{cdiv(P, cand[c].W), gy, 1, cand[c].nthr, cand[c].smem};
    float ms = -1.f;
    for (int r = 0; r < 3; ++r) {
      float t = 0.f;
      if (cudaEventRecord(e0, s) != cudaSuccess || launch_zform<T>(az, g.form, lz, s) != cudaSuccess ||
          cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
        cudaGetLastError();   // a shape the device cannot launch is skipped
        ms = -1.f;
        break;
      }
      if (r > 0 && (ms < 0 || t < ms)) ms = t;
    }
    if (ms >= 0 && (best < 0 || ms < best_ms)) {
      best = (int)c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return NS3D_ERR_CUDA;
  set_form_tile(&g, cand[best]);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_form_tile[key] = best;
  return NS3D_OK;
}

int autotune_padded_size(int N, ns3d_dtype dtype, const ns3d_params& prm, cudaStream_t s) {
  const std::vector<int> cand = pad_candidates(N);
  if (cand.size() < 2 || register_kernels_at(N, cand[0], dtype)) return cand[0];
  int dev = 0;
  cudaDeviceProp pr{};
  std::string name = "unknown";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&pr, dev) == cudaSuccess)
    name = pr.name;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_cache_load();
  const auto key = std::make_tuple(name, N, (int)dtype);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) return it->second;
  int bestP = cand[0];
  double bestT = -1.0;
  for (int P : cand) {
    const double t = time_rhs(N, P, dtype, prm, s);
    if (t > 0 && (bestT < 0 || t < bestT)) {
      bestT = t;
      bestP = P;
    }
  }
  g_tune[key] = bestP;
  tune_cache_store(name, N, (int)dtype, bestP);
  return bestP;
}

}  // namespace

extern "C" ns3d_status ns3d_plan_create(ns3d_plan* out, const int* N_per_member, int batch,
                                        ns3d_dtype dtype, const ns3d_params* prm,
                                        void* cuda_stream, size_t workspace_limit_bytes) {
  if (!out) return NS3D_ERR_INVALID_ARG;
  *out = nullptr;
  if (!N_per_member || batch <= 0 || (dtype != NS3D_F32 && dtype != NS3D_F64))
    return NS3D_ERR_INVALID_ARG;
  ns3d_params P;
  if (prm) P = *prm;
  else ns3d_params_default(&P);
  if (!(P.L > 0) || !(P.nu >= 0) || !(P.s >= 0.5) || !(P.theta > 0) || !(P.eps0 >= 0) ||
      !(P.mN_coef >= 0) || (P.q_form != 0 && P.q_form != 1) || P.n_pad < -1 ||
      !(P.dt_fixed >= 0) || (P.dt_fixed == 0 && !(P.cfl > 0)))
    return NS3D_ERR_INVALID_ARG;
  if (P.nonlinear_form < 0 || P.nonlinear_form > 2) return NS3D_ERR_INVALID_ARG;
  std::map<int, std::vector<int>> byN;
  for (int i = 0; i < batch; ++i) {
    const int N = N_per_member[i];
    if (N < 4 || N % 2 || N > 4096) return NS3D_ERR_INVALID_ARG;
    byN[N].push_back(i);
  }
  ns3d_plan p = new (std::nothrow) ns3d_plan_s();
  if (!p) return NS3D_ERR_OUT_OF_MEMORY;
  p->dtype = dtype;
  p->esz = dtype == NS3D_F32 ? 8 : 16;
  p->prm = P;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  p->loc.resize(batch);
  size_t need = 0, stag = 0;
  for (auto& kv : byN) {
    Level L;
    L.N = kv.first;
    L.B = (int)kv.second.size();
    L.members = kv.second;
    if (P.n_pad > 0) {
      if (2 * P.n_pad < 3 * L.N) { delete p; return NS3D_ERR_INVALID_ARG; }
      L.P = P.n_pad;
    } else if (P.n_pad == 0 && P.nonlinear_form == 0) {
      if (dtype == NS3D_F32) kernels_init<float>();
      else kernels_init<double>();
      L.P = autotune_padded_size(L.N, dtype, P, p->stream);
    } else {
      L.P = default_padded_size(L.N);
    }
    if (!make_geom(L.N, L.P, p->esz, &L.g) || !set_form_geom(&L.g, P.nonlinear_form)) {
      delete p;
      return NS3D_ERR_NOT_SUPPORTED;
    }
    L.sp = make_spec_params(L.N, L.P, P.L, P.nu, P.s, P.theta, P.eps0, P.mN_coef, P.q_form, P.cfl,
                            P.dt_fixed);
    L.fused = P.nonlinear_form == 0 &&
              (dtype == NS3D_F32 ? xfused_available<float>(L.g) : xfused_available<double>(L.g));
    const Geom& g = L.g;
    need += (size_t)L.B * (2 * g.nU + g.nW1 + g.nW2) * p->esz + (size_t)L.P * p->esz +
            (size_t)L.B * sizeof(Ns3dCtrl);
    stag = std::max(stag, d1_bytes(L.N, p->esz));
    for (int j = 0; j < L.B; ++j) p->loc[kv.second[j]] = {(int)p->levels.size(), j};
    p->levels.push_back(L);
  }
  need += stag;
  if (workspace_limit_bytes && need > workspace_limit_bytes) {
    delete p;
    return NS3D_ERR_OUT_OF_MEMORY;
  }
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return NS3D_ERR_CUDA;
  }
  ns3d_status st = NS3D_OK;
  if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) st = NS3D_ERR_CUDA;
  if (st == NS3D_OK) {
    cudaError_t e = dtype == NS3D_F32 ? kernels_init<float>() : kernels_init<double>();
    if (e != cudaSuccess) st = NS3D_ERR_CUDA;
  }
  for (Level& L : p->levels) {
    if (st != NS3D_OK) break;
    const Geom& g = L.g;
    if ((st = dev_alloc(p, &L.U0, (size_t)L.B * g.nU * p->esz)) != NS3D_OK) break;
    if ((st = dev_alloc(p, &L.US, (size_t)L.B * g.nU * p->esz)) != NS3D_OK) break;
    if ((st = dev_alloc(p, &L.W1, (size_t)L.B * g.nW1 * p->esz)) != NS3D_OK) break;
    if ((st = dev_alloc(p, &L.W2, (size_t)L.B * g.nW2 * p->esz)) != NS3D_OK) break;
    if ((st = dev_alloc(p, &L.twP, (size_t)L.P * p->esz)) != NS3D_OK) break;
    void* c = nullptr;
    if ((st = dev_alloc(p, &c, (size_t)L.B * sizeof(Ns3dCtrl))) != NS3D_OK) break;
    L.ctrl = static_cast<Ns3dCtrl*>(c);
    st = dtype == NS3D_F32 ? upload_twiddles<float>(L, p->stream) : upload_twiddles<double>(L, p->stream);
    if (st != NS3D_OK) break;
    if (g.form != 0 && P.n_pad != -1 && !zform_register(g)) {
      st = dtype == NS3D_F32 ? tune_form_tile<float>(L, dtype, p->stream)
                             : tune_form_tile<double>(L, dtype, p->stream);
      if (st != NS3D_OK) break;
    }
    if (L.fused && !xfused_make_maps(&L.maps, g, L.B, L.W2, L.U0, L.US)) L.fused = false;
    if ((st = dev_alloc(p, &L.lamT, lambda_entries(g) * p->esz / 2)) != NS3D_OK) break;
    st = dtype == NS3D_F32 ? upload_lambda<float>(L, p->stream) : upload_lambda<double>(L, p->stream);
    if (st != NS3D_OK) break;
    if (cudaMemsetAsync(L.U0, 0, (size_t)L.B * g.nU * p->esz, p->stream) != cudaSuccess ||
        cudaMemsetAsync(L.US, 0, (size_t)L.B * g.nU * p->esz, p->stream) != cudaSuccess ||
        launch_ctrl_reset(L.ctrl, L.B, p->stream) != cudaSuccess)
      st = NS3D_ERR_CUDA;
  }
  if (st == NS3D_OK) st = dev_alloc(p, &p->staging, stag);
  if (st == NS3D_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) st = NS3D_ERR_CUDA;
  if (st != NS3D_OK) {
    free_all(p);
    delete p;
    return st;
  }
  p->staging_bytes = stag;
  p->launches_per_step = 0;
  for (const Level& L : p->levels) p->launches_per_step += L.g.form ? 22 : (L.fused ? 13 : 19);
  *out = p;
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_plan_destroy(ns3d_plan p) {
  if (!p) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  cudaStreamSynchronize(p->stream);
  free_all(p);
  delete p;
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_plan_info(ns3d_plan p, int member, int* N, int* P, size_t* bytes,
                                      int* launches) {
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  if (N) *N = L->N;
  if (P) *P = L->P;
  if (bytes) *bytes = p->bytes;
  if (launches) *launches = p->launches_per_step;
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_set_initial(ns3d_plan p, int member, const void* uhat, int on_device) {
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  if (!uhat) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  if (p->dtype == NS3D_F32)
    st = put_d1<float>(p, *L, uhat, on_device, static_cast<cplx<float>*>(L->U0) + idx * L->g.nU);
  else
    st = put_d1<double>(p, *L, uhat, on_device, static_cast<cplx<double>*>(L->U0) + idx * L->g.nU);
  if (st != NS3D_OK) return st;
  NS3D_CK(launch_ctrl_reset(L->ctrl + idx, 1, p->stream));
  NS3D_CK(launch_ctrl_set_tend(L->ctrl + idx, 1, p->t_end, p->stream));
  L->a_valid = false;
  if (!on_device) NS3D_CK(cudaStreamSynchronize(p->stream));
  return NS3D_OK;
}

namespace {

// Leray projection (I - kappa kappa^T / |kappa|^2) of one member's state in the
// compact layout [3][kx N][ky N][kz h]; k = 0 is left as it is (the mean flow)
template <typename T>
__global__ void k_project(cplx<T>* u, int N, T kscale) {
  const int h = N / 2;
  const long long plane = (long long)N * N * h;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x) {
    const int kz = (int)(i % h), ky = (int)((i / h) % N), kx = (int)(i / ((long long)N * h));
    const T k0 = kscale * T(kx < h ? kx : kx - N), k1 = kscale * T(ky < h ? ky : ky - N),
            k2 = kscale * T(kz);
    const T kk = k0 * k0 + k1 * k1 + k2 * k2;
    if (!(kk > T(0))) continue;
    const cplx<T> a = u[i], b = u[plane + i], c = u[2 * plane + i];
    const T dr = (k0 * a.x + k1 * b.x + k2 * c.x) / kk, di = (k0 * a.y + k1 * b.y + k2 * c.y) / kk;
    u[i] = cmake(a.x - k0 * dr, a.y - k0 * di);
    u[plane + i] = cmake(b.x - k1 * dr, b.y - k1 * di);
    u[2 * plane + i] = cmake(c.x - k2 * dr, c.y - k2 * di);
  }
}

}  // namespace

extern "C" ns3d_status ns3d_project(ns3d_plan p, int member) {
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  DeviceGuard dg(p->device);
  const long long plane = (long long)L->g.N * L->g.N * L->g.h;
  const int grid = (int)std::min<long long>((plane + 255) / 256, 152 * 8);
  if (p->dtype == NS3D_F32)
    k_project<float><<<grid, 256, 0, p->stream>>>(static_cast<cplx<float>*>(L->U0) + idx * L->g.nU,
                                                   L->g.N, (float)L->sp.kscale);
  else
    k_project<double><<<grid, 256, 0, p->stream>>>(static_cast<cplx<double>*>(L->U0) + idx * L->g.nU,
                                                    L->g.N, L->sp.kscale);
  NS3D_CK(cudaGetLastError());
  L->a_valid = false;
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_get_state(ns3d_plan p, int member, void* out, int on_device,
                                      double* t_out) {
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  if (!out) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  if (p->dtype == NS3D_F32)
    st = get_d1<float>(p, *L, static_cast<const cplx<float>*>(L->U0) + idx * L->g.nU, out, on_device);
  else
    st = get_d1<double>(p, *L, static_cast<const cplx<double>*>(L->U0) + idx * L->g.nU, out, on_device);
  if (st != NS3D_OK) return st;
  Ns3dCtrl c;
  NS3D_CK(cudaMemcpyAsync(&c, L->ctrl + idx, sizeof(c), cudaMemcpyDeviceToHost, p->stream));
  NS3D_CK(cudaStreamSynchronize(p->stream));
  if (t_out) *t_out = c.t;
  return status_of_flags(c.status);
}

extern "C" ns3d_status ns3d_get_clock(ns3d_plan p, int member, double* t, int* nsteps) {
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  if (!t || !nsteps) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  Ns3dCtrl c;
  NS3D_CK(cudaMemcpyAsync(&c, L->ctrl + idx, sizeof(c), cudaMemcpyDeviceToHost, p->stream));
  NS3D_CK(cudaStreamSynchronize(p->stream));
  *t = c.t;
  *nsteps = c.nsteps;
  return status_of_flags(c.status);
}

extern "C" ns3d_status ns3d_set_clock(ns3d_plan p, int member, double t, int nsteps) {
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  if (!(t >= 0.0) || nsteps < 0) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  NS3D_CK(launch_ctrl_set_clock(L->ctrl + idx, t, nsteps, p->stream));
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_step(ns3d_plan p, int nsteps, double t_end) {
  NvtxRange nvtx_("ns3d_step");
  if (!p || nsteps < 0) return NS3D_ERR_INVALID_ARG;
  if (nsteps == 0) return NS3D_OK;
  DeviceGuard dg(p->device);
  if (t_end != p->t_end) {
    for (Level& L : p->levels) NS3D_CK(launch_ctrl_set_tend(L.ctrl, L.B, t_end, p->stream));
    p->t_end = t_end;
  }
  ns3d_status st = ensure_prologue(p);
  if (st != NS3D_OK) return st;
  st = build_graph(p);
  if (st != NS3D_OK) return st;
  for (int i = 0; i < nsteps; ++i) NS3D_CK(cudaGraphLaunch(p->exec, p->stream));
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_synchronize(ns3d_plan p) {
  if (!p) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  NS3D_CK(cudaStreamSynchronize(p->stream));
  int flags = 0;
  for (Level& L : p->levels) {
    std::vector<Ns3dCtrl> c(L.B);
    NS3D_CK(cudaMemcpy(c.data(), L.ctrl, L.B * sizeof(Ns3dCtrl), cudaMemcpyDeviceToHost));
    for (const Ns3dCtrl& x : c) flags |= x.status;
  }
  return status_of_flags(flags);
}

extern "C" ns3d_status ns3d_eval_rhs(ns3d_plan p, int member, const void* uhat, void* rhs,
                                     int on_device) {
  NvtxRange nvtx_("ns3d_eval_rhs");
  Level* L;
  int idx;
  ns3d_status st = member_lookup(p, member, &L, &idx);
  if (st != NS3D_OK) return st;
  if (!uhat || !rhs) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  if (p->dtype == NS3D_F32) {
    cplx<float>* slot = static_cast<cplx<float>*>(L->US) + idx * L->g.nU;
    if ((st = put_d1<float>(p, *L, uhat, on_device, slot)) != NS3D_OK) return st;
    if ((st = enqueue_stage<float>(*L, 0, idx, 1, slot, slot, false, p->stream)) != NS3D_OK) return st;
    if ((st = get_d1<float>(p, *L, slot, rhs, on_device)) != NS3D_OK) return st;
  } else {
    cplx<double>* slot = static_cast<cplx<double>*>(L->US) + idx * L->g.nU;
    if ((st = put_d1<double>(p, *L, uhat, on_device, slot)) != NS3D_OK) return st;
    if ((st = enqueue_stage<double>(*L, 0, idx, 1, slot, slot, false, p->stream)) != NS3D_OK) return st;
    if ((st = get_d1<double>(p, *L, slot, rhs, on_device)) != NS3D_OK) return st;
  }
  L->a_valid = false;   // the evaluation used W1
  if (!on_device) NS3D_CK(cudaStreamSynchronize(p->stream));
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_test_poison_workspaces(ns3d_plan p) {
  if (!p) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  for (Level& L : p->levels) {
    const Geom& g = L.g;
    NS3D_CK(cudaMemsetAsync(L.W1, 0xFF, (size_t)L.B * g.nW1 * p->esz, p->stream));
    NS3D_CK(cudaMemsetAsync(L.W2, 0xFF, (size_t)L.B * g.nW2 * p->esz, p->stream));
    NS3D_CK(cudaMemsetAsync(L.US, 0xFF, (size_t)L.B * g.nU * p->esz, p->stream));
    L.a_valid = false;   // W1 no longer holds the x-inverse of the state
  }
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_test_stall_staging(ns3d_plan p, int on) {
  if (!p) return NS3D_ERR_INVALID_ARG;
  bool any = false;
  for (Level& L : p->levels) {
    if (!L.fused) continue;
    L.extra_tx = on ? 16u : 0u;
    any = true;
  }
  if (!any) return NS3D_ERR_NOT_SUPPORTED;
  DeviceGuard dg(p->device);
  NS3D_CK(cudaStreamSynchronize(p->stream));
  if (p->exec) cudaGraphExecDestroy(p->exec);   // rebuilt with the new launch arguments
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  return NS3D_OK;
}

extern "C" ns3d_status ns3d_step_timed(ns3d_plan p, int nsteps, double t_end, double* kernel_ms,
                                       int* launches) {
  NvtxRange nvtx_("ns3d_step_timed");
  if (!p || nsteps < 0 || !kernel_ms || !launches) return NS3D_ERR_INVALID_ARG;
  DeviceGuard dg(p->device);
  if (t_end != p->t_end) {
    for (Level& L : p->levels) NS3D_CK(launch_ctrl_set_tend(L.ctrl, L.B, t_end, p->stream));
    p->t_end = t_end;
  }
  ns3d_status st = ensure_prologue(p);
  if (st != NS3D_OK) return st;
  KernelTimer tm;
  for (int i = 0; i < 7; ++i) NS3D_CK(cudaEventCreate(&tm.ev[i]));
  for (int n = 0; n < nsteps && st == NS3D_OK; ++n) {
    for (Level& L : p->levels) {
      for (int stage = 1; stage <= 3 && st == NS3D_OK; ++stage) {
        const bool um = stage == 1 && p->prm.dt_fixed <= 0;
        if (p->dtype == NS3D_F32) {
          cplx<float>* U0 = static_cast<cplx<float>*>(L.U0);
          cplx<float>* US = static_cast<cplx<float>*>(L.US);
          st = enqueue_stage<float>(L, stage, 0, L.B, stage == 1 ? U0 : US, stage == 3 ? U0 : US, um,
                                    p->stream, &tm);
        } else {
          cplx<double>* U0 = static_cast<cplx<double>*>(L.U0);
          cplx<double>* US = static_cast<cplx<double>*>(L.US);
          st = enqueue_stage<double>(L, stage, 0, L.B, stage == 1 ? U0 : US, stage == 3 ? U0 : US, um,
                                     p->stream, &tm);
        }
        if (st != NS3D_OK) break;
        if (cudaEventSynchronize(tm.ev[6]) != cudaSuccess) {
          st = NS3D_ERR_CUDA;
          break;
        }
        for (int k = 0; k < 6; ++k) {
          if (L.fused && (k == 0 || k == 4)) continue;   // folded into kind 5
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, tm.ev[k], tm.ev[k + 1]) != cudaSuccess) {
            st = NS3D_ERR_CUDA;
            break;
          }
          kernel_ms[k] += ms;
          launches[k] += 1;
        }
      }
    }
  }
  for (int i = 0; i < 7; ++i) cudaEventDestroy(tm.ev[i]);
  return st;
}

// ------------------------------------------------------------ internal views

namespace {
void fill_view(const Level& L, int index, LevelView* v) {
  v->N = L.N;
  v->P = L.P;
  v->B = L.B;
  v->index = index;
  v->g = &L.g;
  v->U0 = L.U0;
  v->US = L.US;
  v->W1 = L.W1;
  v->W2 = L.W2;
  v->twP = L.twP;
  v->ctrl = L.ctrl;
  v->sp = L.sp;
}
}  // namespace

bool find_level(ns3d_plan p, int N, LevelView* out) {
  if (!p) return false;
  for (size_t i = 0; i < p->levels.size(); ++i)
    if (p->levels[i].N == N) {
      fill_view(p->levels[i], (int)i, out);
      return true;
    }
  return false;
}

bool member_view(ns3d_plan p, int member, LevelView* out, int* idx) {
  Level* L;
  if (member_lookup(p, member, &L, idx) != NS3D_OK) return false;
  fill_view(*L, p->loc[member].first, out);
  return true;
}

cudaStream_t p_stream(ns3d_plan p) { return p->stream; }
ns3d_dtype plan_dtype(ns3d_plan p) { return p->dtype; }
const ns3d_params& plan_params(ns3d_plan p) { return p->prm; }

ns3d_status status_of_level(ns3d_plan p, const LevelView& L) {
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return NS3D_ERR_CUDA;
  std::vector<Ns3dCtrl> c(L.B);
  if (cudaMemcpy(c.data(), L.ctrl, L.B * sizeof(Ns3dCtrl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return NS3D_ERR_CUDA;
  int flags = 0;
  for (const Ns3dCtrl& x : c) flags |= x.status;
  return status_of_flags(flags);
}

PlanDeviceGuard::PlanDeviceGuard(ns3d_plan p) {
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (p && prev != p->device) cudaSetDevice(p->device);
}

PlanDeviceGuard::~PlanDeviceGuard() {
  int cur = -1;
  if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}
