/*
 * ns3d.h - C ABI of the GB300 spectral hyper-viscosity solver for the 3D
 * incompressible Navier-Stokes / Euler equations on the periodic torus.
 *
 * Method (Rohner & Mishra, "Efficient Computation of Large-Scale Statistical
 * Solutions to Incompressible Fluid Flows", PASC'24):
 *   - spatial discretisation: eq. shv_disc (section 2.2) with the Fourier
 *     multiplier Q_N and the scalings m_N ~ N^theta, eps_N ~ N^(1-2s);
 *   - Fourier-space evolution with the pressure eliminated by the Leray
 *     projection (section 2.3), d/dt u_k = (I - k k^T/|k|^2) b_k,
 *     b_k = -i k^T . F[u (x) u]_k, computed by Algorithm 2 (pad to >= 3N/2,
 *     inverse FFT, product, forward FFT, remove the upper third, derivative);
 *   - axis-by-axis padding fused with the transforms (Algorithm 3, section 3.2);
 *   - SSP-RK3 time stepping (section 2.3, eq. RK3);
 *   - Monte Carlo ensembles and their statistics (Algorithm 1, section 2.1;
 *     writers, section 2.4).
 *
 * Conventions shared by every call
 * --------------------------------
 * Fourier coefficients ("D1 layout"): for a member of resolution N (even),
 *   complex array [3][N][N][N/2+1], index [component][kx][ky][kz], kz fastest,
 *   wavenumber k = i for i < N/2 and i - N otherwise (x, y), kz = 0..N/2,
 *   u_hat_k = N^-3 sum_x u(x) exp(-i kappa.x), kappa = (2 pi / L) k,
 *   u(x) = sum over the full spectrum of u_hat_k exp(i kappa.x).
 * Element type: interleaved complex of the plan's dtype (NS3D_F32: 2 floats,
 *   NS3D_F64: 2 doubles).  Only the retained modes |k_i| <= N/2 - 1 are kept
 *   (the projection P_N of eq. shv_disc): Nyquist planes are ignored on input
 *   and returned as zero.
 * Pointers: "on_device" arguments say whether a pointer is device memory of
 *   the plan's GPU (non-zero) or host memory (zero).  The caller owns every
 *   buffer it passes; device buffers must stay valid until the plan's stream
 *   has passed the call.  The plan owns all workspaces it allocates.
 * Streams: every call is ordered on the CUDA stream given at plan creation;
 *   calls with host buffers synchronise that stream before returning.
 * Errors: every call returns an ns3d_status and never aborts.  Conditions
 *   found on the device (a non-finite velocity, lambda_max * dt above the
 *   SSP-RK3 stability limit 2.5) are sticky per member and reported by the
 *   next call that synchronises (ns3d_synchronize, ns3d_get_state,
 *   ns3d_ensemble_stats).
 */
#ifndef NS3D_H
#define NS3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns3d_plan_s* ns3d_plan;

typedef enum {
  NS3D_OK = 0,
  NS3D_ERR_INVALID_ARG = 1,    /* bad size, index, pointer or parameter */
  NS3D_ERR_OUT_OF_MEMORY = 2,  /* workspace above the limit, or cudaMalloc failed */
  NS3D_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  NS3D_ERR_NONFINITE = 4,      /* a member's velocity became NaN/Inf */
  NS3D_ERR_UNSTABLE_DT = 5,    /* lambda_max * dt > 2.5 for some member */
  NS3D_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
  NS3D_ERR_NOT_SUPPORTED = 7   /* e.g. a padded size with a prime factor > 7 */
} ns3d_status;

typedef enum { NS3D_F32 = 0, NS3D_F64 = 1 } ns3d_dtype;

/* Parameters of eq. shv_disc and of the time step.
 *   lambda_k = nu |kappa|^2 + eps_N |kappa|^(2s) Q_k   (damping of mode k)
 *   eps_N = eps0 * N^(1-2s),  m_N = mN_coef * N^theta
 *   Q_k = 0 for |k| <= m_N, else 1 - (m_N/|k|)^((2s-1)/theta) (q_form 0) or 1 (q_form 1)
 *   (|k| the integer wavenumber; the paper's "+eps_N" is read as damping).
 *   n_pad: padded FFT size P.  0: chosen at plan creation (section 3.1): the
 *          smallest 2^a 3^b 5^c 7^d >= 3N/2 where the register kernels exist
 *          (FP32, P = 3N/2 in {48, 96, 192, 384, 1536}; FP64, P = 3N/2 in
 *          {192, 384, 1152}, transformed in double-single arithmetic with a
 *          48-bit significand, binary64 in memory), otherwise the fastest
 *          of the 7-smooth sizes up to 12.5% above it by a timed right-hand
 *          side (cached per device, N and dtype; also in the file named by the
 *          environment variable NS3D_AUTOTUNE_CACHE, if set).  -1: the
 *          smallest such size without a benchmark.  > 0: that size (values
 *          below 3N/2 alias and are rejected).
 *   nonlinear_form: the nonlinear term b before the Leray projection.
 *          0 = divergence form -i k.F[u (x) u] (the paper's, section 2.3):
 *          3 inverse and 6 forward transforms per evaluation, the fused FP32
 *          kernels.  1 = advective form -F[(u . grad) u] from u and its nine
 *          derivatives: 12 inverse and 3 forward.  2 = rotational form
 *          F[u x curl u]: 6 inverse and 3 forward.  For a divergence-free
 *          field with 3/2 padding the three agree after the projection up to
 *          rounding.  Forms 1 and 2 take the smallest 7-smooth padded size
 *          when n_pad = 0 (no benchmark) and need more workspace (form 1:
 *          twice that of form 0); their z pass is a register-resident kernel
 *          in FP32 at P = 3N/2 in {48, 96, 192, 384}, otherwise a tile kernel
 *          whose tile shape plan creation times and picks (n_pad = -1 keeps a
 *          fixed shape).
 *          ns3d_eval_rhs_noalloc takes form 0 only.
 *   dt_fixed > 0: fixed time step; otherwise dt = cfl * (L/N) / max_x sum_i |u_i|
 *          evaluated on the padded grid of the stage-1 field, per member. */
typedef struct {
  double L;
  double nu;
  double s;
  double theta;
  double eps0;
  double mN_coef;
  int q_form;
  int n_pad;
  int nonlinear_form;
  double cfl;
  double dt_fixed;
} ns3d_params;

/* Fills *p with L = 2 pi, nu = 0, s = 1.5, theta = 0.5, eps0 = 1, mN_coef = 1,
 * q_form = 0, n_pad = 0, nonlinear_form = 0, cfl = 0.5, dt_fixed = 0. */
void ns3d_params_default(ns3d_params* p);

/* Creates a plan for an ensemble of `batch` members (Algorithm 1), member i of
 * resolution N_per_member[i] (even, >= 4).  Members of equal N form one level
 * and advance together.  dtype selects the arithmetic of the whole path.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) of the current
 * device.  workspace_limit_bytes: 0 = no limit; otherwise the plan fails with
 * NS3D_ERR_OUT_OF_MEMORY before allocating if it would need more.
 * Members start at u = 0, t = 0.  Errors: INVALID_ARG (sizes, params, null),
 * NOT_SUPPORTED (padded size not 7-smooth, or a form-1/2 z tile of one column
 * that does not fit in shared memory: FP64 P > 1446 (form 1) or > 1808
 * (form 2), FP32 P > 2854 (form 1) or > 3568 (form 2)),
 * OUT_OF_MEMORY, CUDA. */
ns3d_status ns3d_plan_create(ns3d_plan* out, const int* N_per_member, int batch, ns3d_dtype dtype,
                             const ns3d_params* p, void* cuda_stream,
                             size_t workspace_limit_bytes);

/* Releases every device resource of the plan (synchronises its stream). */
ns3d_status ns3d_plan_destroy(ns3d_plan plan);

/* Describes the plan: padded size P of `member`'s level, bytes of device
 * memory the plan holds, and number of kernels one ns3d_step launches. */
ns3d_status ns3d_plan_info(ns3d_plan plan, int member, int* N, int* P, size_t* device_bytes,
                           int* launches_per_step);

/* Sets member `member`'s coefficients (D1 layout, plan dtype) and resets its
 * time to 0 (initial data u(0) = P_N u0 of eq. shv_disc). */
ns3d_status ns3d_set_initial(ns3d_plan plan, int member, const void* uhat, int uhat_on_device);

/* Replaces member `member`'s state by its divergence-free part, the Leray
 * projection (I - kappa kappa^T / |kappa|^2) u_hat_k of section 2.3 at every
 * k != 0 (the mean flow k = 0 is kept): for initial data that is not
 * divergence-free, such as the perturbed Taylor-Green and shear-flow measures
 * of section 6, whose evolution starts from the projected field.  The clock is
 * unchanged.  Stream-ordered. */
ns3d_status ns3d_project(ns3d_plan plan, int member);

/* Copies member `member`'s coefficients out (D1 layout, Nyquist planes zero)
 * and, if t_out is not NULL, its time.  Synchronises; returns the member's
 * sticky device status (NONFINITE / UNSTABLE_DT) if one was raised. */
ns3d_status ns3d_get_state(ns3d_plan plan, int member, void* uhat_out, int out_on_device,
                           double* t_out);

/* Member `member`'s clock: the time reached and the number of completed
 * steps.  Synchronises; returns the member's sticky device status like
 * ns3d_get_state. */
ns3d_status ns3d_get_clock(ns3d_plan plan, int member, double* t, int* nsteps);

/* Sets member `member`'s clock (t >= 0, nsteps >= 0), e.g. after
 * ns3d_set_initial restored a checkpointed state: the run then continues
 * exactly as if it had not stopped (the same steps, clipped at the same
 * t_end).  Stream-ordered. */
ns3d_status ns3d_set_clock(ns3d_plan plan, int member, double t, int nsteps);

/* Advances every member by `nsteps` SSP-RK3 steps (eq. RK3; three evaluations
 * of Algorithm 2 each).  t_end > 0: a member's step is clipped so it stops at
 * t_end exactly, and members already at t_end do not move.  Asynchronous: the
 * work is a CUDA graph replayed on the plan's stream. */
ns3d_status ns3d_step(ns3d_plan plan, int nsteps, double t_end);

/* Waits for the plan's stream and returns the first sticky device status of
 * any member (NS3D_OK if none). */
ns3d_status ns3d_synchronize(ns3d_plan plan);

/* Evaluates the time derivative d/dt u_hat = R(u_hat) of section 2.3
 * (Algorithm 2) for one field of member `member`'s resolution, without
 * touching the member's state.  uhat in and rhs_out in D1 layout. */
ns3d_status ns3d_eval_rhs(ns3d_plan plan, int member, const void* uhat, void* rhs_out,
                          int on_device);

/* Discrete adjoint of one SSP-RK3 step (not in the paper; the exact transpose
 * of eq. RK3 and of the linearised right-hand side of section 2.3 in the real
 * inner product <a,b> = Re sum_k conj(a_k) b_k over the full spectrum).
 * Given the forward state uhat_n at the start of the step and the adjoint
 * lambda_np1 of the state after it, writes lambda_n = (d u_{n+1}/d u_n)^T
 * lambda_np1.  The stages are recomputed from uhat_n.  The step uses the
 * plan's dt_fixed (must be > 0; dt does not depend on u).  All arrays D1
 * layout, plan dtype, device or host per on_device.  Member's state unchanged. */
ns3d_status ns3d_adjoint_step(ns3d_plan plan, int member, const void* lambda_np1, void* lambda_n,
                              const void* uhat_n, int on_device);

/* Gradient of the band energy J = 1/2 sum_{k_lo <= |k| < k_hi} |u_hat_k(T)|^2
 * (full spectrum) after nsteps fixed steps of dt_fixed, with respect to the
 * member's current state u_hat(0), by the discrete adjoint.
 *   checkpoint_every = C > 0: the forward pass keeps every C-th state; the
 *     backward pass recomputes one segment of C steps at a time from its
 *     checkpoint, keeping the three stage states of each of its steps (device
 *     memory: ceil(nsteps/C) + 3C states).
 *   checkpoint_every <= 0: the forward pass keeps the three stage states of
 *     every step and nothing is recomputed (3 nsteps states: 75 MB per step
 *     at 128^3 FP32, 600 MB at 256^3), the fastest form where HBM allows.
 * Either way the result is the same to rounding.  grad_uhat0 in D1 layout.
 * The member's state is unchanged.  Errors: NOT_SUPPORTED (dt_fixed <= 0),
 * OUT_OF_MEMORY (the kept states do not fit), INVALID_ARG. */
ns3d_status ns3d_grad_band_energy(ns3d_plan plan, int member, double k_lo, double k_hi,
                                  int nsteps, int checkpoint_every, void* grad_uhat0,
                                  int on_device);

/* The observable of ns3d_grad_band_energy at member `member`'s current state:
 * J = 1/2 sum_{k_lo <= |k| < k_hi} |u_hat_k|^2 over the full spectrum (the
 * energy of a band of shells, here the end-time observable whose gradient the
 * discrete adjoint gives; not in the paper, which defines the energy
 * spectrum of section 2.4).  Summed in FP64 with compensation in a fixed
 * order (reproducible bit for bit) and written to the host double *J.
 * Synchronises; returns the member's sticky device status like
 * ns3d_get_state.  Errors: INVALID_ARG (null, k_hi <= k_lo, bad member). */
ns3d_status ns3d_band_energy(ns3d_plan plan, int member, double k_lo, double k_hi, double* J);

/* Ensemble statistics of the members of resolution level_N at their current
 * state (writers of section 2.4; Algorithm 1 step 3), accumulated in FP64 on
 * the device.  Every array is host memory owned by the caller; any pointer may
 * be NULL to skip that output.
 *   mean          [3][N][N][N]  sample mean of u_i at the N^3 grid points x_j = j L/N
 *   second        [6][N][N][N]  sample mean of u_i u_j (order 00 01 02 11 12 22)
 *   var           [3][N][N][N]  sample variance of u_i (divisor M-1; 0 if M = 1)
 *   spectrum      [N]           mean of E(K) = 1/2 sum_{round|k| = K} |u_hat_k|^2
 *   spectrum_se   [N]           its Monte Carlo standard error sqrt(var/M)
 *   s2, s2_se     [N/2]         mean and standard error of
 *                               S2(r) = (1/3) sum_d <|u(x + r e_d) - u(x)|^2>, r = jL/N
 *   energy, energy_se           mean and standard error of E = 1/2 <|u|^2>
 *   members                     M, the number of members of the level
 *   enstrophy_spectrum[_se] [N] mean and standard error of
 *                               Z(K) = 1/2 sum_{round|k| = K} |kappa|^2 |u_hat_k|^2
 *                               (= 1/2 |omega_hat|^2 by shell for divergence-free u)
 *   enstrophy, enstrophy_se     of Z = 1/2 <|omega|^2> = sum_K Z(K)
 *   dissipation, dissipation_se of D = sum_k lambda_k |u_hat_k|^2 over the full
 *                               spectrum: the exact energy loss rate -dE/dt of
 *                               the semi-discrete system (the dealiased
 *                               nonlinear term conserves E)
 *   s2_ball, s2_ball_se [N/2]   mean and standard error of the ball-averaged
 *                               S2_ball(r) = < (1/|B_r|) int_{|h|<=r} |u(x+h) - u(x)|^2 dh >_x
 *                               = sum_k |u_hat_k|^2 2 (1 - 3 (sin q - q cos q) / q^3),
 *                               q = |kappa| r, r = jL/N (computed only when
 *                               either pointer is non-NULL: N/2 passes over the
 *                               coefficients)
 * The spectra, S2 and D are compensated FP64 sums in a fixed order: two calls on
 * the same state return the same bits. */
typedef struct {
  double* mean;
  double* second;
  double* var;
  double* spectrum;
  double* spectrum_se;
  double* s2;
  double* s2_se;
  double energy;
  double energy_se;
  int members;
  double* enstrophy_spectrum;
  double* enstrophy_spectrum_se;
  double enstrophy;
  double enstrophy_se;
  double dissipation;
  double dissipation_se;
  double* s2_ball;
  double* s2_ball_se;
} ns3d_stats;

ns3d_status ns3d_ensemble_stats(ns3d_plan plan, int level_N, ns3d_stats* out);

/* |omega(x)|, the vorticity magnitude of member `member` at the N^3 grid points
 * x_j = j L/N (omega = curl u, from omega_hat = i kappa x u_hat; the paper's
 * vorticity field, section 6.1), as a real array [N][N][N] (z fastest) of the
 * plan dtype in device or host memory per out_on_device.  Synchronises.
 * NOT_SUPPORTED if N has a prime factor above 7. */
ns3d_status ns3d_vorticity_magnitude(ns3d_plan plan, int member, void* out, int out_on_device);

/* The velocity u(x) of member `member` at the N^3 grid points x_j = j L/N
 * (inverse transform of the retained modes), as a real array [3][N][N][N]
 * (z fastest) of the plan dtype in device or host memory per out_on_device:
 * the samples whose one-point marginals the statistics compare across
 * resolutions (section 6.1, mesh refinement).  Synchronises.  NOT_SUPPORTED if
 * N has a prime factor above 7. */
ns3d_status ns3d_physical_field(ns3d_plan plan, int member, void* out, int out_on_device);

/* Mesh-refinement measures of section 6.1 between two levels of the plan: the
 * coarse level of resolution coarse_N (Ma members) and the fine level fine_N
 * (Mb members, fine_N a multiple of coarse_N), compared at the coarse grid
 * points x_j = j L / coarse_N (for the fine fields: their values at those
 * points), per velocity component c, each averaged over the points:
 *   w1[c]          1-point Wasserstein distance of the one-point marginals,
 *                  W1 = integral |F_a(t) - F_b(t)| dt of the empirical CDFs of
 *                  the Ma coarse and Mb fine values at the point
 *   mean_err[c]    |mean_a - mean_b| (sample means)
 *   var_err[c]     |var_a - var_b| (sample variances, divisor M - 1)
 *   sample_err[c]  mean over members m of |a_m - b_m| (member m of each level
 *                  drawn from the same sample of the initial measure); -1 when
 *                  Ma != Mb
 *   mc_se[c]       sqrt(var_a / Ma + var_b / Mb): the Monte Carlo error bar
 *                  of the difference of the means, the floor below which
 *                  mean_err cannot be resolved
 * Sums are compensated FP64 in a fixed order.  The members' fields are formed
 * on the device (as ns3d_physical_field); temporary device memory: (Ma + Mb)
 * x 3 coarse_N^3 values plus one fine field.  Synchronises.  Errors:
 * INVALID_ARG (no such level, fine_N not a multiple of coarse_N),
 * NOT_SUPPORTED (more than 128 members in a level, or N with a prime factor
 * above 7), OUT_OF_MEMORY. */
typedef struct {
  double w1[3];
  double mean_err[3];
  double var_err[3];
  double sample_err[3];
  double mc_se[3];
  int coarse_members;
  int fine_members;
} ns3d_refinement;

ns3d_status ns3d_mesh_refinement(ns3d_plan plan, int coarse_N, int fine_N, ns3d_refinement* out);

/* Diagnostic: advances every member by `nsteps` steps like ns3d_step, but
 * launches the kernels one by one (no graph) with CUDA events recorded on the
 * plan's stream around each of them, and adds the measured milliseconds of
 * each kernel kind to kernel_ms[0..5] and the number of stage evaluations to
 * launches[0..5] (kinds: 0 inverse x, 1 inverse y, 2 fused z pass, 3 forward
 * y, 4 forward x, 5 spectral step; where a level runs the fused x pass -- the
 * forward x, spectral step and next stage's inverse x in one kernel -- its
 * time is under kind 5 and kinds 0 and 4 stay at zero).  Synchronises.  The
 * paper times single kernel calls the same way to compare them with lower
 * bounds (Table 2). */
ns3d_status ns3d_step_timed(ns3d_plan plan, int nsteps, double t_end, double* kernel_ms,
                            int* launches);

/* Allocation-free right-hand side for small grids (the paper has no
 * counterpart; it is a service for callers that may not allocate device
 * memory when they need the derivative: hosts whose device memory budget is
 * fixed at start-up, plug-ins that must not re-enter the host's allocator
 * from a callback, loops that cannot afford cudaMalloc's implicit device
 * synchronisation).  Computes the same R(u_hat) as ns3d_eval_rhs without a
 * plan: uhat and rhs_out are device buffers of the current device in D1
 * layout and `dtype`, all work is enqueued on cuda_stream (a cudaStream_t)
 * and nothing waits.  Every intermediate array lives in one 8 MiB file-scope
 * device array of the library (held by every GPU that loads it until exit);
 * no cudaMalloc or other allocation happens.  Limits: 4 <= N <= 32 and padded
 * size P <= 48, else NS3D_ERR_INVALID_ARG; n_pad 0 or -1 takes the smallest
 * 7-smooth P >= 3N/2, and a given P with a prime factor above 7 returns
 * NS3D_ERR_NOT_SUPPORTED (as ns3d_plan_create does).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; after a cudaDeviceReset of that
 * device this entry point must not be called again.  All calls share the array and it keeps the last
 * call's contents: calls that overlap on the GPU race; order them on one
 * stream. */
ns3d_status ns3d_eval_rhs_noalloc(int N, ns3d_dtype dtype, const ns3d_params* p,
                                  const void* uhat, void* rhs_out, void* cuda_stream);

/* Static text for a status code. */
/* Test hook for the failure path of the bounded device waits (no counterpart
 * in the paper).  While `on` is nonzero, every launch of the fused x pass
 * (FP32 levels with P = 3N/2, P in {48, 96, 192, 384}) expects 16 bytes more
 * on its first staged input tile than the tile's copy delivers, so each
 * block's wait for that tile ends at its time limit (about one second): the
 * block flags its member TIMEOUT, waits (bounded) for its other copies and
 * returns; the member's state is then undefined and the next call that reads
 * the device status returns NS3D_ERR_TIMEOUT.  Nothing faults and the CUDA
 * context stays usable.  Synchronises the plan's stream.  Returns
 * NS3D_ERR_NOT_SUPPORTED if no level of the plan runs the fused pass.  Off by
 * default. */
ns3d_status ns3d_test_stall_staging(ns3d_plan plan, int on);

/* Test hook (no counterpart in the paper): fills every level's workspaces and
 * stage-state buffer with all-ones bytes, a NaN in FP32 and FP64, so that a
 * kernel that reads a workspace element no earlier pass wrote shows up as a
 * NONFINITE status or a wrong result.  The state itself is left alone; the
 * next step re-derives everything it needs from it.  Stream-ordered. */
ns3d_status ns3d_test_poison_workspaces(ns3d_plan plan);

const char* ns3d_status_string(ns3d_status s);

#ifdef __cplusplus
}
#endif

#endif /* NS3D_H */
