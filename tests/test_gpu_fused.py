"""GPU parity of the FP32 fused x pass (forward x of the products, spectral
step, RK3 combine and the next stage's inverse x in one TMA-staged kernel)
against the oracle, through the C ABI.

The fused pass runs for FP32 levels at P = 3N/2 with P in {48, 96, 192,
384}.  It keeps the x-inverse of each member's state in a workspace between
steps, so these tests cover what can make that copy stale: several members
per level (the tile rows of every member), members frozen at t_end, and
state or workspace changes between steps (set_initial, eval_rhs)."""
import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def rel(a, b):
    a = np.asarray(a)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


@pytest.fixture(scope="module")
def B(lib):
    from paper_2401_09843_gb300 import binding
    return binding


def test_fused_levels_with_several_members(B):
    """Three 32^3 and two 64^3 members (two fused levels), per-member CFL
    steps: each evolves as if alone; the plan launches 13 kernels per level
    and step (inverse x folded into the fused pass)."""
    Ns = [32, 64, 32, 64, 32]
    prm = S.Params(cfl=0.4, eps0=1.0, nu=0.005)
    p = B.Plan(Ns, B.NS3D_F32, cfl=0.4, eps0=1.0, nu=0.005)
    assert p.info(0)["launches_per_step"] == 2 * 13
    u0 = [I.random_spectrum(n, seed=11, member=m, k0=3.0) * (1.0 - 0.15 * m)
          for m, n in enumerate(Ns)]
    for m, u in enumerate(u0):
        p.set_initial(m, u)
    p.step(3)
    for m in range(len(Ns)):
        got, t = p.get_state(m, with_time=True)
        ref, tref, _ = S.integrate(u0[m], prm, 3)
        assert abs(t - tref) < 1e-6 * tref, m
        assert rel(got.cpu().numpy(), ref) < TOL32, m
    p.close()


def test_fused_t_end_clipping_and_frozen_members(B):
    N = 32
    prm = S.Params(cfl=0.5, eps0=1.0)
    u0 = I.random_spectrum(N, seed=5, k0=3.0)
    p = B.Plan([N, N], B.NS3D_F32, cfl=0.5, eps0=1.0)
    p.set_initial(0, u0)
    p.set_initial(1, 0.5 * u0)           # slower flow: larger CFL step, fewer steps
    p.step(60, t_end=0.25)
    for m, scale in ((0, 1.0), (1, 0.5)):
        got, t = p.get_state(m, with_time=True)
        assert abs(t - 0.25) < 1e-12
        ref, _, _ = S.integrate(scale * u0, prm, 60, t_end=0.25)
        assert rel(got.cpu().numpy(), ref) < TOL32, m
    before = [p.get_state(m).cpu().numpy() for m in range(2)]
    p.step(3, t_end=0.25)                # at t_end: nothing moves
    for m in range(2):
        assert np.array_equal(p.get_state(m).cpu().numpy(), before[m])
    # moving t_end on continues from the frozen state (its kept x-inverse)
    p.step(2, t_end=0.3)
    got, t = p.get_state(0, with_time=True)
    ref, tref, _ = S.integrate(before[0].astype(np.complex128), prm, 2, t_end=0.3 - 0.25)
    assert abs((t - 0.25) - tref) < 1e-6
    assert rel(got.cpu().numpy(), ref) < TOL32
    p.close()


def test_fused_state_changes_between_steps(B):
    """eval_rhs reuses the workspace that carries the x-inverse between
    steps, set_initial replaces the state: both must be seen by the next
    step."""
    N = 32
    prm = S.Params(eps0=1.0, dt_fixed=0.004)
    u0 = I.random_spectrum(N, seed=8, k0=3.0)
    u1 = I.random_spectrum(N, seed=9, k0=2.5)
    p = B.Plan([N], B.NS3D_F32, eps0=1.0, dt_fixed=0.004)
    p.set_initial(0, u0)
    p.step(2)
    r = p.eval_rhs(0, u1).cpu().numpy()
    assert rel(r, S.rhs(u1, prm)) < TOL32
    p.step(2)
    ref, _, _ = S.integrate(u0, prm, 4)
    assert rel(p.get_state(0).cpu().numpy(), ref) < TOL32
    p.set_initial(0, u1)
    p.step(1)
    ref, _, _ = S.integrate(u1, prm, 1)
    assert rel(p.get_state(0).cpu().numpy(), ref) < TOL32
    p.close()


def test_fused_mean_flow_and_zero_field(B):
    N = 64
    p = B.Plan([N, N], B.NS3D_F32, eps0=1.0, dt_fixed=0.01)
    u = I.random_spectrum(N, seed=1, k0=3.0)
    u[:, 0, 0, 0] = [0.3, -0.2, 0.1]      # a mean flow is carried unchanged
    p.set_initial(0, u)
    p.set_initial(1, np.zeros_like(u))    # zero stays zero
    p.step(2)
    got = p.get_state(0).cpu().numpy()
    assert np.allclose(got[:, 0, 0, 0], [0.3, -0.2, 0.1], atol=1e-7)
    ref, _, _ = S.integrate(u, S.Params(eps0=1.0, dt_fixed=0.01), 2)
    assert rel(got, ref) < TOL32
    assert np.all(p.get_state(1).cpu().numpy() == 0)
    p.close()


def test_staging_wait_times_out_with_status(B):
    """Failure path of the bounded waits: with the test hook the first
    staged tile never completes; every block gives up after its time limit,
    the step reports TIMEOUT, and the context stays usable (a new plan steps
    correctly).  No fault, trap or endless wait is involved."""
    N = 32
    u0 = I.random_spectrum(N, seed=4, k0=3.0)
    p = B.Plan([N], B.NS3D_F32, eps0=1.0, dt_fixed=0.004)
    p.set_initial(0, u0)
    p.test_stall_staging(True)
    p.step(1)
    with pytest.raises(B.Ns3dError) as e:
        p.synchronize()
    assert e.value.code == 6
    p.close()
    fp64 = B.Plan([N], B.NS3D_F64, eps0=1.0)
    with pytest.raises(B.Ns3dError) as e:
        fp64.test_stall_staging(True)        # no fused level
    assert e.value.code == 7
    fp64.close()
    p = B.Plan([N], B.NS3D_F32, eps0=1.0, dt_fixed=0.004)
    p.set_initial(0, u0)
    p.step(2)
    ref, _, _ = S.integrate(u0, S.Params(eps0=1.0, dt_fixed=0.004), 2)
    assert rel(p.get_state(0).cpu().numpy(), ref) < TOL32
    p.close()
