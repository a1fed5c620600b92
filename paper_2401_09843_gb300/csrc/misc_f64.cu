// Point-wise kernels, double.
#include "kernels_misc.cuh"
NS3D_MISC_VARIANT(double)

namespace ns3d {

__global__ void k_ctrl_reset(Ns3dCtrl* c, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    c[i].t = 0.0;
    c[i].dt = 0.0;
    c[i].t_end = 0.0;
    c[i].umax_bits = 0ull;
    c[i].status = 0;
    c[i].nsteps = 0;
    c[i].dtf = 0.f;
  }
}

__global__ void k_ctrl_set_tend(Ns3dCtrl* c, int n, double t_end) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i].t_end = t_end;
}

__global__ void k_ctrl_set_clock(Ns3dCtrl* c, double t, int nsteps) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->t = t;
    c->nsteps = nsteps;
  }
}

__global__ void k_step_dt(Ns3dCtrl* c, int n, SpecParams sp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) step_dt_member(c[i], sp);
}

cudaError_t launch_step_dt(Ns3dCtrl* c, int n, const SpecParams& sp, cudaStream_t s) {
  k_step_dt<<<(n + 127) / 128, 128, 0, s>>>(c, n, sp);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_reset(Ns3dCtrl* c, int n, cudaStream_t s) {
  k_ctrl_reset<<<(n + 127) / 128, 128, 0, s>>>(c, n);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_set_tend(Ns3dCtrl* c, int n, double t_end, cudaStream_t s) {
  k_ctrl_set_tend<<<(n + 127) / 128, 128, 0, s>>>(c, n, t_end);
  return cudaGetLastError();
}

cudaError_t launch_ctrl_set_clock(Ns3dCtrl* c, double t, int nsteps, cudaStream_t s) {
  k_ctrl_set_clock<<<1, 32, 0, s>>>(c, t, nsteps);
  return cudaGetLastError();
}

}  // namespace ns3d
