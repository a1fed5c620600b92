"""GPU discrete adjoint (ns3d_adjoint_step, ns3d_grad_band_energy) against the
oracle's pinned adjoint, central finite differences of GPU forward runs along
seeded random divergence-free directions, and the autograd wrapper."""
import numpy as np
import pytest

import ns3d_inputs as I
from oracle import adjoint as A
from oracle import solver as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


@pytest.mark.parametrize("N", [12, 16])
def test_adjoint_step_matches_oracle(lib, N):
    from paper_2401_09843_gb300 import binding as B
    dt = 0.04
    prm = S.Params(nu=0.01, eps0=1.0)
    p = B.Plan([N], B.NS3D_F64, nu=0.01, eps0=1.0, dt_fixed=dt)
    u = I.random_spectrum(N, seed=5, k0=2.5)
    lam = I.random_spectrum(N, seed=6, k0=3.0)
    got = p.adjoint_step(0, lam, u).cpu().numpy()
    ref = A.rk3_adjoint_step(u, lam, dt, prm)
    assert rel(got, ref) < 1e-11
    # the transpose of the (oracle) tangent step
    du = I.random_spectrum(N, seed=7, k0=3.0)
    lhs = S.inner(lam, A.rk3_tangent_step(u, du, dt, prm))
    assert abs(S.inner(got, du) - lhs) < 1e-11 * abs(lhs)
    p.close()


@pytest.mark.parametrize("C", [4, 1, 6, 0])
def test_grad_band_energy_matches_oracle(lib, C):
    """Every memory mode: segments of 4 + 2 steps, one step per checkpoint, one
    recomputed segment, and all stage states kept from the forward pass."""
    from paper_2401_09843_gb300 import binding as B
    N, dt, n = 12, 0.04, 6
    prm = S.Params(nu=0.01, eps0=1.0)
    u0 = I.random_spectrum(N, seed=8, k0=2.5)
    p = B.Plan([N], B.NS3D_F64, nu=0.01, eps0=1.0, dt_fixed=dt)
    p.set_initial(0, u0)
    got = p.grad_band_energy(0, 2.0, 4.0, n, checkpoint_every=C).cpu().numpy()
    ref = A.grad_band_energy(u0, prm, n, dt, 2.0, 4.0, checkpoint_every=4)
    assert rel(got, ref) < 1e-11
    assert np.array_equal(p.get_state(0).cpu().numpy(), u0)     # state untouched
    p.close()


def test_grad_band_energy_kept_stages_fp32_match_checkpoints(lib):
    """FP32 at a register-kernel size: the kept-stages gradient equals the
    checkpointed one to FP32 rounding (both run the same kernels; only the
    buffers the stage states live in differ), and zero steps give the band
    mask itself."""
    from paper_2401_09843_gb300 import binding as B
    N, dt, n = 32, 0.01, 12
    u0 = I.random_spectrum(N, seed=31, k0=4.0)
    p = B.Plan([N], B.NS3D_F32, eps0=1.0, dt_fixed=dt)
    p.set_initial(0, u0)
    g0 = p.grad_band_energy(0, 4.0, 8.0, n, checkpoint_every=0).cpu().numpy()
    g5 = p.grad_band_energy(0, 4.0, 8.0, n, checkpoint_every=5).cpu().numpy()
    assert rel(g0, g5) < 1e-6
    gz = p.grad_band_energy(0, 4.0, 8.0, 0, checkpoint_every=0).cpu().numpy()
    ref = A.grad_band_energy(u0.astype(np.complex128), S.Params(eps0=1.0), 0, dt, 4.0, 8.0)
    assert rel(gz, ref) < 1e-6
    p.close()


def _J_gpu(B, N, dtype, u, nsteps, dt, k_lo, k_hi):
    p = B.Plan([N], dtype, eps0=1.0, dt_fixed=dt)
    p.set_initial(0, u)
    p.step(nsteps)
    uT = p.get_state(0).cpu().numpy().astype(np.complex128)
    p.close()
    return A.band_energy(uT, k_lo, k_hi)


@pytest.mark.parametrize("N,nsteps,C", [(32, 40, 10)])
def test_gradient_central_differences(lib, N, nsteps, C):
    """Band 8 <= |k| < 16 at step `nsteps`, fixed dt, checkpoints every C
    steps: <grad, v> against central differences of GPU FP64 forward runs
    along seeded random divergence-free directions (seeds 1..3)."""
    from paper_2401_09843_gb300 import binding as B
    dt = 0.01
    u0 = I.random_spectrum(N, seed=20240004)
    p = B.Plan([N], B.NS3D_F64, eps0=1.0, dt_fixed=dt)
    p.set_initial(0, u0)
    g = p.grad_band_energy(0, 8.0, 16.0, nsteps, checkpoint_every=C).cpu().numpy()
    p.close()
    for seed in (1, 2, 3):
        v = I.random_spectrum(N, seed=seed, energy=0.5)
        h = 1e-4
        fd = (_J_gpu(B, N, B.NS3D_F64, u0 + h * v, nsteps, dt, 8.0, 16.0)
              - _J_gpu(B, N, B.NS3D_F64, u0 - h * v, nsteps, dt, 8.0, 16.0)) / (2 * h)
        assert abs(S.inner(g, v) - fd) < 1e-6 * abs(fd), seed


def test_fp32_gradient_tracks_fp64(lib):
    from paper_2401_09843_gb300 import binding as B
    N, dt, n = 32, 0.01, 20
    u0 = I.random_spectrum(N, seed=20240004)
    out = {}
    for dt_ in (B.NS3D_F64, B.NS3D_F32):
        p = B.Plan([N], dt_, eps0=1.0, dt_fixed=dt)
        p.set_initial(0, u0)
        out[dt_] = p.grad_band_energy(0, 8.0, 16.0, n, checkpoint_every=5).cpu().numpy().astype(np.complex128)
        p.close()
    assert rel(out[B.NS3D_F32], out[B.NS3D_F64]) < 1e-4


def test_autograd_wrapper(lib):
    import torch
    from paper_2401_09843_gb300 import binding as B
    from paper_2401_09843_gb300.autograd import band_energy
    N, dt, n = 16, 0.02, 5
    u0 = I.random_spectrum(N, seed=3, k0=3.0)
    x = torch.tensor(u0, dtype=torch.complex128, device="cuda", requires_grad=True)
    J = band_energy(x, 2.0, 5.0, n, dt, eps0=1.0)
    (gx,) = torch.autograd.grad(J, x)
    prm = S.Params(eps0=1.0)
    Jref = A.band_energy(S.integrate(u0, prm.with_(dt_fixed=dt), n)[0], 2.0, 5.0)
    assert abs(J.item() - Jref) < 1e-12 * Jref
    g = A.grad_band_energy(u0, prm, n, dt, 2.0, 5.0)
    w = S.half_weights(N)
    assert rel(gx.cpu().numpy(), g * w) < 1e-11
    # torch's convention: dJ = sum Re(conj(grad) dz) over the stored tensor
    v = I.random_spectrum(N, seed=9, k0=3.0)
    lhs = float(np.sum((np.conj(gx.cpu().numpy()) * v).real))
    assert abs(lhs - S.inner(g, v)) < 1e-11 * abs(lhs)


def test_gradient_config4_size(lib):
    """The adjoint at its stated workload: 128^3 FP64, J = band energy
    8 <= |k| < 16 at step 200, checkpoints every 20 steps, against central
    differences of GPU forward runs along 8 seeded random divergence-free
    directions (seeds 1..8)."""
    from paper_2401_09843_gb300 import binding as B
    N, nsteps, C, dt = 128, 200, 20, 0.005
    u0 = I.random_spectrum(N, seed=20240004)
    p = B.Plan([N], B.NS3D_F64, eps0=1.0, dt_fixed=dt)
    p.set_initial(0, u0)
    g = p.grad_band_energy(0, 8.0, 16.0, nsteps, checkpoint_every=C).cpu().numpy()
    p.close()
    for seed in range(1, 9):
        v = I.random_spectrum(N, seed=seed, energy=0.5)
        h = 2e-5      # O(h^2) truncation ~2e-7 relative here; round-off ~1e-10
        fd = (_J_gpu(B, N, B.NS3D_F64, u0 + h * v, nsteps, dt, 8.0, 16.0)
              - _J_gpu(B, N, B.NS3D_F64, u0 - h * v, nsteps, dt, 8.0, 16.0)) / (2 * h)
        assert abs(S.inner(g, v) - fd) < 1e-6 * abs(fd), seed


@pytest.mark.parametrize("dt,tol", [("f64", 1e-14), ("f32", 1e-14)])
def test_band_energy_observable(lib, dt, tol):
    """ns3d_band_energy against the oracle's J on the member's state, for a
    band that cuts through shells, the whole spectrum (J = E) and an empty
    band; two calls return the same bits."""
    from paper_2401_09843_gb300 import binding as B
    N = 32
    u = I.random_spectrum(N, seed=31, k0=4.0)
    p = B.Plan([N, N], B.NS3D_F64 if dt == "f64" else B.NS3D_F32, eps0=1.0, dt_fixed=0.01)
    p.set_initial(1, u)
    ref_u = p.get_state(1).cpu().numpy().astype(np.complex128)   # the state as stored (FP32 rounded)
    for lo, hi in ((2.5, 7.0), (0.0, 1e9), (100.0, 200.0)):
        J = p.band_energy(1, lo, hi)
        Jref = A.band_energy(ref_u, lo, hi)
        assert abs(J - Jref) <= tol * max(Jref, 1e-300), (lo, hi, J, Jref)
        assert p.band_energy(1, lo, hi) == J
    assert abs(p.band_energy(1, 0.0, 1e9) - S.energy(ref_u)) < 1e-14 * S.energy(ref_u)
    assert p.band_energy(0, 0.0, 1e9) == 0.0          # member 0 is still zero
    with pytest.raises(B.Ns3dError):
        p.band_energy(1, 5.0, 5.0)
    p.close()


@pytest.mark.parametrize("N", [32, 64, 128])
def test_fp32_adjoint_step_register_z_pass(lib, N):
    """FP32 adjoint step at the register sizes P = 3N/2 (48, 96, 192: the
    adjoint's z pass runs register-resident there) against the oracle's
    discrete adjoint, and the transpose identity against its tangent step."""
    from paper_2401_09843_gb300 import binding as B
    dt = 0.01
    prm = S.Params(nu=0.01, eps0=1.0)
    p = B.Plan([N], B.NS3D_F32, nu=0.01, eps0=1.0, dt_fixed=dt)
    assert p.info(0)["P"] == 3 * N // 2
    u = I.random_spectrum(N, seed=50 + N, k0=3.0)
    lam = I.random_spectrum(N, seed=60 + N, k0=4.0)
    got = p.adjoint_step(0, lam, u).cpu().numpy().astype(np.complex128)
    ref = A.rk3_adjoint_step(u, lam, dt, prm)
    assert rel(got, ref) < 2e-5, rel(got, ref)
    du = I.random_spectrum(N, seed=70 + N, k0=3.0)
    lhs = S.inner(lam, A.rk3_tangent_step(u, du, dt, prm))
    assert abs(S.inner(got, du) - lhs) < 2e-5 * abs(lhs)
    p.close()
