"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances: relative L2 over the retained modes <= 1e-11 in FP64 and
<= 2e-5 in FP32 (short horizons; the flow is chaotic beyond them).
Sizes: small grids span several column tiles and ragged tails (N = 24: 12
kz columns in 16-wide tiles; P = 36 in 8-wide z tiles; odd P = 15 and 35,
radices 5 and 7); the full 256^3 size runs in the bench's launch
configuration against the Galerkin product summed mode pair by mode pair
(sparse spectra) and against properties that hold at any size."""
import math

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-11, 2e-5


def rel(a, b):
    a = np.asarray(a)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


@pytest.fixture(scope="module")
def B(lib):
    from paper_2401_09843_gb300 import binding
    return binding


def plan(B, Ns, dtype, **kw):
    return B.Plan(Ns, dtype, **kw)


# --------------------------------------------------------------------------- RHS

@pytest.mark.parametrize("N", [4, 8, 10, 16, 22, 24, 32, 40, 64])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_rhs_matches_oracle(B, N, dt):
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    prm = S.Params(nu=0.01, eps0=1.0, L=5.0)
    uh = I.random_spectrum(N, seed=100 + N, k0=2.5)
    p = plan(B, [N], dtype, nu=0.01, eps0=1.0, L=5.0)
    got = p.eval_rhs(0, uh).cpu().numpy()
    ref = S.rhs(uh, prm)
    assert rel(got, ref) < (TOL64 if dt == "f64" else TOL32)
    # Nyquist planes and the stored kz = N/2 column come back zero
    h = N // 2
    assert np.all(got[:, h] == 0) and np.all(got[:, :, h] == 0) and np.all(got[..., h] == 0)
    p.close()


def test_rhs_q_step_form_and_explicit_padding(B):
    N = 16
    prm = S.Params(nu=0.0, eps0=3.0, s=2.0, theta=0.4, q_form=1, n_pad=32)
    uh = I.random_spectrum(N, seed=2, k0=3.0)
    p = plan(B, [N], B.NS3D_F64, nu=0.0, eps0=3.0, s=2.0, theta=0.4, q_form=1, n_pad=32)
    assert p.info(0)["P"] == 32
    assert rel(p.eval_rhs(0, uh).cpu().numpy(), S.rhs(uh, prm)) < TOL64
    p.close()


@pytest.mark.parametrize("N", [128, 256])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_rhs_full_size_sparse_spectrum(B, N, dt):
    """Full-size grids in the production launch shapes against the truncated
    product summed over mode pairs (no transform on the oracle side)."""
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    prm = S.Params(nu=0.0, eps0=1.0)
    uh = I.sparse_random(N, seed=N + 7, nmodes=48)
    ref = S.rhs_by_convolution(uh, prm)
    p = plan(B, [N], dtype, nu=0.0, eps0=1.0)
    got = p.eval_rhs(0, uh).cpu().numpy()
    assert rel(got, ref) < (TOL64 if dt == "f64" else TOL32)
    p.close()


def test_rhs_full_size_invariants(B):
    """Dense random field at 256^3: inviscid energy and helicity are
    conserved by the RHS, R is divergence-free and Hermitian on kz = 0."""
    N = 256
    uh = I.random_spectrum(N, seed=20240001)
    p = plan(B, [N], B.NS3D_F32, nu=0.0, eps0=0.0)
    R = p.eval_rhs(0, uh).cpu().numpy().astype(np.complex128)
    p.close()
    scale = math.sqrt(S.inner(uh, uh) * S.inner(R, R))
    assert abs(S.inner(uh, R)) < 2e-6 * scale
    w = S.curl(uh, S.TWO_PI)
    assert abs(S.inner(w, R)) < 2e-6 * math.sqrt(S.inner(w, w) * S.inner(R, R))
    assert S.divergence_ratio(R, S.TWO_PI) < 1e-6
    pl = R[:, :, :, 0]
    mirror = np.conj(pl[:, (-np.arange(N)) % N][:, :, (-np.arange(N)) % N])
    assert np.max(np.abs(pl - mirror)) < 1e-5 * np.max(np.abs(pl))


# --------------------------------------------------------------------------- steps

def test_taylor_green_32_fp64_100_steps(B):
    """N = 32^3 Taylor-Green, nu = 0.01 plus the hyper-viscosity for N, fixed
    dt = 0.01: GPU and oracle field by field at steps 1, 10 and 100."""
    N = 32
    prm = S.Params(nu=0.01, eps0=1.0, dt_fixed=0.01)
    u0 = I.taylor_green(N)
    p = plan(B, [N], B.NS3D_F64, nu=0.01, eps0=1.0, dt_fixed=0.01)
    p.set_initial(0, u0)
    ref = u0
    done = 0
    for n in (1, 10, 100):
        p.step(n - done)
        ref, _, _ = S.integrate(ref, prm, n - done)
        done = n
        got, t = p.get_state(0, with_time=True)
        assert rel(got.cpu().numpy(), ref) < TOL64, n
        assert abs(t - 0.01 * n) < 1e-12
    p.close()


def test_taylor_green_32_fp32_steps(B):
    N = 32
    prm = S.Params(nu=0.01, eps0=1.0, dt_fixed=0.01)
    u0 = I.taylor_green(N)
    p = plan(B, [N], B.NS3D_F32, nu=0.01, eps0=1.0, dt_fixed=0.01)
    p.set_initial(0, u0)
    p.step(10)
    ref, _, _ = S.integrate(u0, prm, 10)
    assert rel(p.get_state(0).cpu().numpy(), ref) < TOL32
    p.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_random_ic_cfl_steps(B, dt):
    """CFL time steps: the GPU takes the same dt sequence as the oracle."""
    N = 32
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    prm = S.Params(cfl=0.5, eps0=1.0)
    u0 = I.random_spectrum(N, seed=20240001)
    p = plan(B, [N], dtype, cfl=0.5, eps0=1.0)
    p.set_initial(0, u0)
    p.step(5)
    got, t = p.get_state(0, with_time=True)
    ref, tref, _ = S.integrate(u0, prm, 5, P=p.info(0)["P"])   # the CFL max is taken on the padded grid
    assert abs(t - tref) < (1e-13 if dt == "f64" else 1e-6) * tref
    assert rel(got.cpu().numpy(), ref) < (TOL64 if dt == "f64" else TOL32)
    p.close()


def test_uneven_batch_matches_individual_runs(B):
    """Members of several resolutions in one plan (levels) each evolve as if
    alone; per-member CFL steps differ."""
    Ns = [16, 24, 16, 12, 24]
    prm = S.Params(cfl=0.4, eps0=1.0, nu=0.005)
    p = plan(B, Ns, B.NS3D_F64, cfl=0.4, eps0=1.0, nu=0.005)
    u0 = [I.random_spectrum(n, seed=7, member=m, k0=2.0) for m, n in enumerate(Ns)]
    for m, u in enumerate(u0):
        p.set_initial(m, u)
    p.step(3)
    for m, n in enumerate(Ns):
        got, t = p.get_state(m, with_time=True)
        ref, tref, _ = S.integrate(u0[m], prm, 3, P=p.info(m)["P"])
        assert abs(t - tref) < 1e-13
        assert rel(got.cpu().numpy(), ref) < TOL64, m
    p.close()


def test_t_end_clipping_and_frozen_members(B):
    N = 16
    prm = S.Params(cfl=0.5, eps0=1.0)
    u0 = I.random_spectrum(N, seed=5, k0=2.0)
    p = plan(B, [N, N], B.NS3D_F64, cfl=0.5, eps0=1.0)
    p.set_initial(0, u0)
    p.set_initial(1, 0.5 * u0)           # slower flow: larger CFL step
    p.step(60, t_end=0.25)
    for m, scale in ((0, 1.0), (1, 0.5)):
        got, t = p.get_state(m, with_time=True)
        assert abs(t - 0.25) < 1e-14
        ref, tref, _ = S.integrate(scale * u0, prm, 60, t_end=0.25, P=p.info(m)["P"])
        assert abs(tref - 0.25) < 1e-14
        assert rel(got.cpu().numpy(), ref) < TOL64
    before = p.get_state(0).cpu().numpy()
    p.step(3, t_end=0.25)                # at t_end: nothing moves
    assert np.array_equal(p.get_state(0).cpu().numpy(), before)
    p.close()


def test_host_buffers_and_determinism(B):
    N = 24
    u0 = I.random_spectrum(N, seed=9, k0=3.0)
    outs = []
    for _ in range(2):
        p = plan(B, [N], B.NS3D_F32, eps0=1.0)
        p.set_initial_host(0, u0)
        p.step(4)
        outs.append(p.get_state_host(0)[0])
        p.close()
    assert np.array_equal(outs[0], outs[1])


def test_zero_field_and_mean_flow(B):
    N = 16
    p = plan(B, [N], B.NS3D_F64, eps0=1.0, dt_fixed=0.01)
    z = np.zeros((3, N, N, N // 2 + 1), complex)
    assert np.all(p.eval_rhs(0, z).cpu().numpy() == 0)
    u = I.random_spectrum(N, seed=1, k0=2.0)
    u[:, 0, 0, 0] = [0.3, -0.2, 0.1]      # a mean flow is carried unchanged
    p.set_initial(0, u)
    p.step(2)
    got = p.get_state(0).cpu().numpy()
    assert np.allclose(got[:, 0, 0, 0], [0.3, -0.2, 0.1], atol=1e-15)
    ref, _, _ = S.integrate(u, S.Params(eps0=1.0, dt_fixed=0.01), 2)
    assert rel(got, ref) < TOL64
    p.close()


def test_device_status_nonfinite_and_unstable(B):
    N = 16
    u = I.random_spectrum(N, seed=1, k0=2.0)
    bad = u.copy()
    bad[0, 1, 2, 3] = np.nan
    p = plan(B, [N], B.NS3D_F64, eps0=1.0)
    p.set_initial(0, bad)
    p.step(1)
    with pytest.raises(B.Ns3dError) as e:
        p.synchronize()
    assert e.value.code == 4
    p.close()
    p = plan(B, [N], B.NS3D_F64, eps0=1.0, nu=1.0, dt_fixed=1.0)   # lambda_max dt >> 2.5
    p.set_initial(0, u)
    p.step(1)
    with pytest.raises(B.Ns3dError) as e:
        p.synchronize()
    assert e.value.code == 5
    p.close()


@pytest.mark.parametrize("N,val", [(64, np.nan), (256, np.inf)])
def test_device_status_nonfinite_fp32_register_kernels(B, N, val):
    """FP32 at the register-resident sizes (z pass with the in-register CFL
    maximum, fused x pass): a non-finite coefficient sets NONFINITE."""
    u = I.random_spectrum(N, seed=2, k0=3.0)
    u[2, 3, 1, 5] = val
    p = plan(B, [N], B.NS3D_F32, eps0=1.0)
    p.set_initial(0, u)
    p.step(1)
    with pytest.raises(B.Ns3dError) as e:
        p.synchronize()
    assert e.value.code == 4
    p.close()


def test_workspace_limit_is_enforced(B):
    with pytest.raises(B.Ns3dError) as e:
        B.Plan([64], B.NS3D_F32, workspace_limit=1 << 20)
    assert e.value.code == 2


def test_fp32_path_tracks_fp64_at_256(B):
    """Config-2 workload (256^3 random field, CFL 0.5, hyper-viscosity for N):
    the FP32 path stays within 2e-5 of the FP64 path over 10 steps (the FP64
    path is pinned to the oracle above, at this size by the sparse test)."""
    N = 256
    u0 = I.random_spectrum(N, seed=20240001)
    res = {}
    for dt in (B.NS3D_F64, B.NS3D_F32):
        p = plan(B, [N], dt, eps0=1.0, cfl=0.5)
        p.set_initial(0, u0)
        p.step(1)
        a = p.get_state(0).cpu().numpy().astype(np.complex128)
        p.step(9)
        b, t = p.get_state(0, with_time=True)
        res[dt] = (a, b.cpu().numpy().astype(np.complex128), t)
        p.close()
    assert rel(res[B.NS3D_F32][0], res[B.NS3D_F64][0]) < TOL32
    assert rel(res[B.NS3D_F32][1], res[B.NS3D_F64][1]) < TOL32
    assert abs(res[B.NS3D_F32][2] - res[B.NS3D_F64][2]) < 1e-6 * res[B.NS3D_F64][2]


def test_cufft_comparison_pipeline_matches_oracle(B):
    """The cuFFT pipeline the bench times for comparison computes the same RHS
    (so the comparison times the same work)."""
    import torch
    import bench
    N = 32
    prm = S.Params(eps0=1.0)
    uh = I.random_spectrum(N, seed=3, k0=3.0)
    rhs = bench.cufft_pipeline(torch, N)
    got = rhs(torch.from_numpy(uh).to("cuda", torch.complex64)).cpu().numpy()
    assert rel(got, S.rhs(uh, prm)) < TOL32


@pytest.mark.parametrize("N,dt", [(64, "f32"), (24, "f32"), (32, "f64"), (256, "f32")])
def test_no_kernel_reads_unwritten_workspace(B, N, dt):
    """Workspaces and the stage buffer NaN-filled before the run and again
    between steps: every element a pass reads was written by an earlier pass,
    so the result is bit for bit that of a clean plan (and matches the
    oracle), and no NONFINITE is raised."""
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    prm = S.Params(eps0=1.0, dt_fixed=0.002)
    u0 = I.random_spectrum(N, seed=N + 2, k0=3.0)
    out = []
    for poison in (False, True):
        p = plan(B, [N, N], dtype, eps0=1.0, dt_fixed=0.002)
        if poison:
            p.test_poison_workspaces()
        p.set_initial(0, u0)
        p.set_initial(1, 0.5 * u0)
        p.step(1)
        if poison:
            p.test_poison_workspaces()
        p.step(1)
        p.synchronize()
        r = p.eval_rhs(1, 0.5 * u0)
        if poison:
            p.test_poison_workspaces()
        r2 = p.eval_rhs(1, 0.5 * u0)
        out.append((p.get_state(0).cpu().numpy(), r.cpu().numpy(), r2.cpu().numpy()))
        p.close()
    (s0, r0, _), (s1, r1, r12) = out
    assert np.array_equal(s0, s1) and np.array_equal(r0, r1) and np.array_equal(r1, r12)
    if N <= 64:
        ref, _, _ = S.integrate(u0, prm, 2)
        assert rel(s1, ref) < (TOL64 if dt == "f64" else TOL32)


def test_padded_size_autotune(B):
    """n_pad = 0 times a right-hand side at the 7-smooth sizes within 12.5% of
    3N/2 where no register kernel exists and keeps the fastest; the result is
    the same Galerkin truncation (matches the oracle).  Register-kernel sizes
    and n_pad = -1 take the smallest size."""
    N = 24
    uh = I.random_spectrum(N, seed=5, k0=3.0)
    prm = S.Params(eps0=1.0)
    p = plan(B, [N], B.NS3D_F64, eps0=1.0)
    assert p.info(0)["P"] in (36, 40)
    assert rel(p.eval_rhs(0, uh).cpu().numpy(), S.rhs(uh, prm)) < TOL64
    p.close()
    p = plan(B, [N], B.NS3D_F64, eps0=1.0, n_pad=-1)
    assert p.info(0)["P"] == 36
    p.close()
    p = plan(B, [64], B.NS3D_F32, eps0=1.0)
    assert p.info(0)["P"] == 96
    p.close()


def test_autotune_cache_file(tmp_path):
    """The autotune result is appended to NS3D_AUTOTUNE_CACHE and read back
    by the next process."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2401_09843_gb300 import binding as B\n"
            "p = B.Plan([26], B.NS3D_F64, eps0=1.0)\n"
            "print(p.info(0)['P'])\n" % root)
    env = dict(os.environ, NS3D_AUTOTUNE_CACHE=str(cache))
    P1 = int(subprocess.run([sys.executable, "-c", code], env=env, check=True,
                            stdout=subprocess.PIPE, text=True).stdout.split()[-1])
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[1].split() == ["26", "1", str(P1)]
    P2 = int(subprocess.run([sys.executable, "-c", code], env=env, check=True,
                            stdout=subprocess.PIPE, text=True).stdout.split()[-1])
    assert P2 == P1 and len(cache.read_text().splitlines()) == 1


@pytest.mark.parametrize("N", [32, 256])
def test_fp64_three_pass_z_pass(B, N):
    """FP64 at P = 3N/2 (the three-pass register z pass where it exists):
    sparse RHS against the Galerkin product, and CFL steps at N = 32."""
    prm = S.Params(nu=0.0, eps0=1.0)
    uh = I.sparse_random(N, seed=N + 9, nmodes=40)
    p = plan(B, [N], B.NS3D_F64, nu=0.0, eps0=1.0, n_pad=3 * N // 2)
    assert rel(p.eval_rhs(0, uh).cpu().numpy(), S.rhs_by_convolution(uh, prm)) < TOL64
    p.close()


def test_fp32_and_fp64_statistics_over_500_steps(B):
    """The 256^3 workload over its full horizon (500 CFL steps): pointwise
    agreement is lost to chaos, the energy, enstrophy and dissipation of the
    FP32 run stay within 1% of the FP64 run's and the spectrum within 5% on
    the energetic shells K <= 32."""
    N, n = 256, 500
    u0 = I.random_spectrum(N, seed=20240001)
    st = {}
    for dt in (B.NS3D_F64, B.NS3D_F32):
        p = plan(B, [N], dt, eps0=1.0, cfl=0.5)
        p.set_initial(0, u0)
        p.step(n)
        st[dt] = p.ensemble_stats(N, fields=False)
        assert p.clock(0)[1] == n
        p.close()
    a, b = st[B.NS3D_F32], st[B.NS3D_F64]
    for k in ("energy", "enstrophy", "dissipation"):
        assert abs(a[k] - b[k]) < 1e-2 * b[k], k
    sa, sb = np.asarray(a["spectrum"])[1:33], np.asarray(b["spectrum"])[1:33]
    assert np.max(np.abs(sa - sb) / sb) < 5e-2


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_project_state_matches_oracle_leray(B, dt):
    """ns3d_project leaves the divergence-free part of a member's state (the
    perturbed Taylor-Green data of section 6.1 are not divergence-free) and
    keeps the mean flow; other members are untouched."""
    N = 24
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    u = I.perturbed_taylor_green(N, seed=5, member=1)
    u[:, 0, 0, 0] = [0.1, -0.2, 0.3]
    p = plan(B, [N, N], dtype, L=1.0)
    p.set_initial(0, u)
    p.set_initial(1, u)
    p.project(0)
    got = p.get_state(0).cpu().numpy().astype(np.complex128)
    ref = S.leray(u, 1.0)
    ref[:, 0, 0, 0] = u[:, 0, 0, 0]
    ref = ref * S.retained_mask(N)
    assert rel(got, ref) < (1e-14 if dt == "f64" else 1e-6)
    assert S.divergence_ratio(got, 1.0) < (1e-14 if dt == "f64" else 1e-6)
    other = p.get_state(1).cpu().numpy().astype(np.complex128)
    assert rel(other, u * S.retained_mask(N)) < (1e-15 if dt == "f64" else 1e-7)
    p.close()
