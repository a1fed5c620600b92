"""GPU parity of the production time step against the oracle at the sizes the
throughput is measured at, through the C ABI (ns3d_step).

The plans below are created exactly like the benchmark's (n_pad = 0), so
they run its kernels: in FP32 at 256^3 (P = 384) and 128^3 (P = 192) the
register-resident z pass, the register column passes and the fused x pass
(forward x + spectral step + SSP-RK3 combine + the next stage's inverse x,
13 launches per step); in FP64 the kernels the plan picks for that size.

* 128^3, dense random field: the state after steps 1 and 10 against the
  oracle's padded-transform steps (its per-component transforms spread over
  a spawn-started process pool so ten steps take minutes, not most of an hour).
* 256^3, sparse random field: one whole SSP-RK3 step against the oracle's
  step composed from the mode-pair Galerkin sum (each stage's support grows
  by pair sums: 10 modes become about 4e5); no transform on the oracle side.
* 256^3, ABC Beltrami field moved to shell 100: its projected nonlinear term
  vanishes, so n fixed-dt steps multiply it by r(-lambda dt)^n exactly.

Tolerances: relative L2 over the whole state <= 2e-5 (FP32) and 1e-11
(FP64).  The increment u+ - u is also compared, at 1e-4 (FP32: the FP32
rounding of u itself, about 6e-8 |u|, is then at most 1e-5 of an increment of
1% of u) and 1e-10 (FP64), so that a wrong stage weight cannot hide behind
the unchanged part of the state."""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-11}
TOL_INC = {"f32": 1e-4, "f64": 1e-10}


def rel(a, b):
    a = np.asarray(a)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


@pytest.fixture(scope="module")
def B(lib):
    from paper_2401_09843_gb300 import binding
    return binding


def dtype_of(B, dt):
    return B.NS3D_F32 if dt == "f32" else B.NS3D_F64


# --------------------------------------------------------------------------- 128^3 dense

DENSE_N, DENSE_DT = 128, 4e-3
DENSE_PRM = S.Params(nu=0.0, eps0=1.0, dt_fixed=DENSE_DT)


@pytest.fixture(scope="module")
def dense_reference():
    """Oracle states of the 128^3 random-spectrum field after 1 and 10 steps
    (P = 192, the plans' padded size)."""
    u0 = I.random_spectrum(DENSE_N, seed=20240041)
    workers = min(6, mp.cpu_count())
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        old = S.set_map(ex.map)
        try:
            u1, _, _ = S.integrate(u0, DENSE_PRM, 1, P=3 * DENSE_N // 2)
            u10, _, _ = S.integrate(u1, DENSE_PRM, 9, P=3 * DENSE_N // 2)
        finally:
            S.set_map(old)
    return u0, {1: u1, 10: u10}


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_dense_128_steps_1_and_10(B, dense_reference, dt):
    u0, ref = dense_reference
    p = B.Plan([DENSE_N], dtype_of(B, dt), nu=0.0, eps0=1.0, dt_fixed=DENSE_DT)
    info = p.info(0)
    if dt == "f32":
        assert info["P"] == 192 and info["launches_per_step"] == 13   # the fused path
    p.set_initial(0, u0)
    done = 0
    for n in (1, 10):
        p.step(n - done)
        done = n
        got, t = p.get_state(0, with_time=True)
        got = got.cpu().numpy().astype(np.complex128)
        assert abs(t - n * DENSE_DT) < 1e-12
        assert rel(got, ref[n]) < TOL[dt], (n, rel(got, ref[n]))
        assert rel(got - u0, ref[n] - u0) < TOL_INC[dt], (n, rel(got - u0, ref[n] - u0))
    p.close()


# --------------------------------------------------------------------------- 256^3 sparse

SPARSE_N, SPARSE_DT = 256, 3e-3
SPARSE_PRM = S.Params(nu=0.0, eps0=1.0, dt_fixed=SPARSE_DT)


@pytest.fixture(scope="module")
def sparse_reference():
    """One oracle SSP-RK3 step of a 10-mode field (|k_i| < 48) at 256^3, each
    stage's right-hand side the Galerkin sum over mode pairs."""
    u0 = I.sparse_random(SPARSE_N, seed=20240011, nmodes=10, kmax=48)
    un, _ = S.rk3_step(u0, SPARSE_PRM, rhs_fn=lambda v: S.rhs_by_convolution(v, SPARSE_PRM))
    return u0, un


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_sparse_256_one_step(B, sparse_reference, dt):
    u0, ref = sparse_reference
    nz = np.count_nonzero(np.any(ref != 0, axis=0))
    assert nz > 1e5                               # the step reaches most of the band
    p = B.Plan([SPARSE_N], dtype_of(B, dt), nu=0.0, eps0=1.0, dt_fixed=SPARSE_DT)
    info = p.info(0)
    if dt == "f32":
        assert info["P"] == 384 and info["launches_per_step"] == 13   # the benchmarked path
    p.test_poison_workspaces()                    # every workspace read must have been written
    p.set_initial(0, u0)
    p.step(1)
    got = p.get_state(0).cpu().numpy().astype(np.complex128)
    p.close()
    assert rel(got, ref) < TOL[dt], rel(got, ref)
    assert rel(got - u0, ref - u0) < TOL_INC[dt], rel(got - u0, ref - u0)


# --------------------------------------------------------------------------- 256^3 Beltrami

@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_beltrami_shell_100_steps_256(B, dt):
    """An ABC field's coefficients do not depend on its shell: taken at |k| = 5
    and moved to |k| = 100 (hyper-viscous range, m_N = 16), 20 fixed steps
    must give r(-lambda dt)^20 times the initial field exactly."""
    N, Kshell, nsteps, step_dt = 256, 100, 20, 2e-3
    K, V = I.modes_of(I.beltrami_abc(16, K=5), rtol=1e-12)
    K = K * (Kshell // 5)
    u0 = np.zeros((3, N, N, N // 2 + 1), dtype=np.complex128)
    u0[:, K[:, 0] % N, K[:, 1] % N, K[:, 2]] = V.T
    prm = S.Params(nu=0.0, eps0=1.0, dt_fixed=step_dt)
    lam = float(S.dissipation_of_k2(np.array([Kshell * Kshell]), N, prm)[0])
    assert lam * step_dt > 0.01
    r = S.rk3_amplification(-lam * step_dt) ** nsteps
    p = B.Plan([N], dtype_of(B, dt), nu=0.0, eps0=1.0, dt_fixed=step_dt)
    p.set_initial(0, u0)
    p.step(nsteps)
    got = p.get_state(0).cpu().numpy().astype(np.complex128)
    p.close()
    assert rel(got, r * u0) < TOL[dt], rel(got, r * u0)
