"""Full-size grids of the largest workloads (1024^3 FP32, P = 1536; 768^3
FP64, P = 1152) through the C ABI, in the launch shapes the plan uses there
(arrays of up to 7e9 complex elements per member: 64-bit offsets throughout).

The inputs are built on the device from mode lists, so the host never holds
a dense field of these sizes (and the workspaces are NaN-filled first, so a
read of an element no pass wrote would show): a sparse random field against the oracle's
mode-pair Galerkin sum (rhs_sparse), and an ABC Beltrami field whose
projected nonlinear term vanishes, so that n fixed-dt RK3 steps multiply it
by r(-lambda_K dt)^n exactly (r the RK3 stability polynomial)."""
import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-11}


@pytest.fixture(scope="module")
def B(lib):
    from paper_2401_09843_gb300 import binding
    return binding


def on_device(torch, K, V, N, cdtype):
    u = torch.zeros((3, N, N, N // 2 + 1), dtype=cdtype, device="cuda")
    ix = torch.from_numpy(K[:, 0] % N).cuda()
    iy = torch.from_numpy(K[:, 1] % N).cuda()
    iz = torch.from_numpy(K[:, 2]).cuda()
    u[:, ix, iy, iz] = torch.from_numpy(np.ascontiguousarray(V.T)).to("cuda", cdtype)
    return u, (ix, iy, iz)


def release(torch):
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("N,dt", [(1024, "f32"), (768, "f64")])
def test_rhs_largest_grids_sparse_field(B, N, dt):
    import torch
    dtype = B.NS3D_F32 if dt == "f32" else B.NS3D_F64
    cdt = torch.complex64 if dt == "f32" else torch.complex128
    prm = S.Params(nu=0.0, eps0=1.0)
    K, V = I.sparse_modes(N, seed=N + 5, nmodes=40)
    assert np.max(np.abs(K[:, :2])) > N // 2 - 64     # modes near the band edge
    Ko, Rref = S.rhs_sparse(K, V, N, prm)
    # P = 3N/2 explicitly: the three-pass register z kernels of both precisions
    p = B.Plan([N], dtype, nu=0.0, eps0=1.0, n_pad=3 * N // 2)
    p.test_poison_workspaces()          # every workspace read must have been written
    u, _ = on_device(torch, K, V, N, cdt)
    R = p.eval_rhs(0, u)
    p.synchronize()
    del u
    ox, oy, oz = (torch.from_numpy(a).cuda() for a in (Ko[:, 0] % N, Ko[:, 1] % N, Ko[:, 2]))
    got = R[:, ox, oy, oz].T.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - Rref) < TOL[dt] * np.linalg.norm(Rref)
    # and nothing anywhere else
    total = float(torch.sum(torch.abs(R.to(torch.complex128)) ** 2))
    assert abs(total - float(np.sum(np.abs(got) ** 2))) < 2 * TOL[dt] * total
    p.close()
    del R
    release(torch)


@pytest.mark.parametrize("N,dt,nsteps", [(1024, "f32", 3), (768, "f64", 2)])
def test_beltrami_steps_largest_grids(B, N, dt, nsteps):
    import torch
    dtype = B.NS3D_F32 if dt == "f32" else B.NS3D_F64
    cdt = torch.complex64 if dt == "f32" else torch.complex128
    # an ABC field's coefficients do not depend on its shell: take them at
    # |k| = 5 and move the wave vectors to |k| = 200, deep in the range where
    # the hyper-viscosity acts (m_N = N^(1/2)); nu = 0 keeps lambda_max dt
    # below the RK3 limit at these N
    Kshell = 200
    K, V = I.modes_of(I.beltrami_abc(16, K=5), rtol=1e-12)
    assert len(K) == 5
    K = K * (Kshell // 5)
    prm = S.Params(nu=0.0, eps0=1.0, dt_fixed=2e-3)
    lam = float(S.dissipation_of_k2(np.array([Kshell * Kshell]), N, prm)[0])
    assert lam * prm.dt_fixed > 0.01
    r = S.rk3_amplification(-lam * prm.dt_fixed) ** nsteps
    p = B.Plan([N], dtype, nu=0.0, eps0=1.0, dt_fixed=2e-3)
    p.test_poison_workspaces()          # every workspace read must have been written
    u, (ix, iy, iz) = on_device(torch, K, V, N, cdt)
    p.set_initial(0, u)
    p.step(nsteps)
    got, t = p.get_state(0, with_time=True)
    del u
    assert abs(t - nsteps * 2e-3) < 1e-15
    at = got[:, ix, iy, iz].T.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(at - r * V) < TOL[dt] * np.linalg.norm(r * V)
    total = float(torch.sum(torch.abs(got.to(torch.complex128)) ** 2))
    assert abs(total - float(np.sum(np.abs(at) ** 2))) < 2 * TOL[dt] * total
    p.close()
    del got
    release(torch)
