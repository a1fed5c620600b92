"""GPU ensemble statistics (ns3d_ensemble_stats) against the oracle's
definitions, and agreement of evolved ensembles within Monte Carlo error bars."""
import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S
from oracle import stats as T
from paper_2401_09843_gb300.ensemble import merge_stats

pytestmark = pytest.mark.gpu

KEYS = [("mean", "mean"), ("second", "second"), ("var", "var"), ("spectrum", "spectrum"),
        ("spectrum_se", "spectrum_stderr"), ("s2", "s2"), ("s2_se", "s2_stderr"),
        ("enstrophy_spectrum", "enstrophy_spectrum"),
        ("enstrophy_spectrum_se", "enstrophy_spectrum_stderr"),
        ("s2_ball", "s2_ball"), ("s2_ball_se", "s2_ball_stderr")]
SCALARS = ["energy", "enstrophy", "dissipation"]


def _check(gpu, ref, rtol):
    for gk, rk in KEYS:
        a, b = np.asarray(gpu[gk]), np.asarray(ref[rk])
        assert np.max(np.abs(a - b)) <= rtol * max(np.max(np.abs(b)), 1e-30), gk
    for k in SCALARS:
        if k not in ref:
            continue
        assert abs(gpu[k] - ref[k]) <= rtol * ref[k], k
        assert abs(gpu[k + "_se"] - ref[k + "_stderr"]) <= rtol * max(ref[k], 1e-30), k
    assert gpu["members"] == ref["M"]


@pytest.mark.parametrize("dt,rtol", [("f64", 1e-11), ("f32", 2e-6)])
def test_stats_match_oracle(lib, dt, rtol):
    from paper_2401_09843_gb300 import binding as B
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    Ns = [16, 8, 16, 16, 8, 16, 16]          # two levels; the N = 16 level has 5 members
    p = B.Plan(Ns, dtype, eps0=1.0, nu=0.01)
    prm = S.Params(eps0=1.0, nu=0.01)
    u = [I.random_spectrum(n, seed=41, member=m, k0=2.5) for m, n in enumerate(Ns)]
    for m, x in enumerate(u):
        p.set_initial(m, x)
    for N in (16, 8):
        mem = [m for m, n in enumerate(Ns) if n == N]
        ref = T.ensemble_stats(np.stack([u[m] for m in mem]), S.TWO_PI, prm)
        _check(p.ensemble_stats(N), ref, rtol)
    # the vorticity magnitude field of one member
    w = p.vorticity_magnitude(0).cpu().numpy()
    wref = T.vorticity_magnitude(u[0], S.TWO_PI)
    assert np.max(np.abs(w - wref)) <= rtol * np.max(wref)
    p.close()


def test_perturbed_taylor_green_energy_budget(lib):
    """The paper's perturbed Taylor-Green workload (section 6.1: unit torus,
    s = 1.5, 8 x 3 uniform first-harmonic perturbations per sample) as an
    ensemble: the energy writer's time series obeys dE/dt = -D with D the
    dissipation writer (trapezoidal in time, error O(dt^3) per step), the
    enstrophy writer matches the oracle, and the vorticity field is finite."""
    from paper_2401_09843_gb300 import binding as B
    N, M, dt, nsteps = 32, 4, 2e-4, 10
    prm = S.Params(L=1.0, eps0=1.0, nu=1e-3, dt_fixed=dt)
    p = B.Plan([N] * M, B.NS3D_F64, L=1.0, eps0=1.0, nu=1e-3, dt_fixed=dt)
    # the perturbations are drawn per component; the flow starts from their
    # divergence-free part (the solver evolves P u0)
    u = [S.leray(I.perturbed_taylor_green(N, seed=601, member=m), 1.0) for m in range(M)]
    for m, x in enumerate(u):
        p.set_initial(m, x)
    series = [p.ensemble_stats(N, fields=False)]
    for _ in range(nsteps):
        p.step(1)
        series.append(p.ensemble_stats(N, fields=False))
    for a, b in zip(series[:-1], series[1:]):
        dE = b["energy"] - a["energy"]
        assert abs(dE + 0.5 * dt * (a["dissipation"] + b["dissipation"])) < 1e-5 * abs(dE)
    uT = [S.integrate(x, prm, nsteps)[0] for x in u]
    ref = T.ensemble_stats(np.stack(uT), 1.0, prm)
    last = series[-1]
    assert abs(last["enstrophy"] - ref["enstrophy"]) < 1e-11 * ref["enstrophy"]
    assert abs(last["dissipation"] - ref["dissipation"]) < 1e-11 * ref["dissipation"]
    assert np.max(np.abs(np.asarray(last["enstrophy_spectrum"]) - ref["enstrophy_spectrum"])) \
        < 1e-11 * np.max(ref["enstrophy_spectrum"])
    w = p.vorticity_magnitude(0).cpu().numpy()
    assert np.all(np.isfinite(w)) and np.max(np.abs(w - T.vorticity_magnitude(uT[0], 1.0))) \
        < 1e-10 * np.max(w)
    p.close()


def test_single_member_has_zero_errors(lib):
    from paper_2401_09843_gb300 import binding as B
    p = B.Plan([12], B.NS3D_F64, eps0=1.0)
    u = I.random_spectrum(12, seed=2)
    p.set_initial(0, u)
    st = p.ensemble_stats(12)
    assert st["members"] == 1 and np.all(st["var"] == 0) and np.all(st["spectrum_se"] == 0)
    assert abs(st["energy"] - S.energy(u)) < 1e-14
    p.close()


def test_evolved_ensemble_within_error_bars_and_shard_merge(lib):
    """8 random members evolved 5 CFL steps in FP32 on the GPU and in FP64 by
    the oracle: statistics agree within 3 combined Monte Carlo standard
    errors (here far closer: the same members); two 'virtual ranks' of 4
    members merge (Chan) to the 8-member statistics."""
    from paper_2401_09843_gb300 import binding as B
    N, M = 16, 8
    u = [I.random_spectrum(N, seed=77, member=m, k0=3.0) for m in range(M)]
    prm = S.Params(eps0=1.0, cfl=0.5)
    p = B.Plan([N] * M, B.NS3D_F32, eps0=1.0, cfl=0.5)
    for m in range(M):
        p.set_initial(m, u[m])
    p.step(5)
    g = p.ensemble_stats(N)
    ref = T.ensemble_stats(np.stack([S.integrate(x, prm, 5)[0] for x in u]), S.TWO_PI)
    comb = np.sqrt(np.asarray(g["spectrum_se"]) ** 2 + ref["spectrum_stderr"] ** 2)
    assert np.all(np.abs(np.asarray(g["spectrum"]) - ref["spectrum"]) <= 3 * comb + 1e-12)
    assert abs(g["energy"] - ref["energy"]) <= 3 * np.hypot(g["energy_se"], ref["energy_stderr"])
    halves = []
    for part in (u[:4], u[4:]):
        q = B.Plan([N] * 4, B.NS3D_F32, eps0=1.0, cfl=0.5)
        for m, x in enumerate(part):
            q.set_initial(m, x)
        q.step(5)
        halves.append(q.ensemble_stats(N))
        q.close()
    merged = merge_stats(halves[0], halves[1])
    for k in ("mean", "second", "var", "spectrum", "spectrum_se", "s2", "energy"):
        assert np.allclose(merged[k], g[k], rtol=1e-9, atol=1e-12), k
    p.close()


def test_cylindrical_shear_flow_mean_and_variance(lib):
    """The paper's cylindrical shear flow (section 6.2; unit torus, s = 1.5,
    rho = 0.05, p = 10 perturbation modes of amplitude delta = 0.025) as an
    FP64 ensemble: the pointwise mean and variance of u_x after a few steps
    match the oracle on the same samples, and the domain mean of u_x (the
    k = 0 mode) is carried unchanged."""
    from paper_2401_09843_gb300 import binding as B
    N, M, dt, nsteps = 32, 4, 2e-4, 5
    prm = S.Params(L=1.0, eps0=1.0, dt_fixed=dt)
    p = B.Plan([N] * M, B.NS3D_F64, L=1.0, eps0=1.0, dt_fixed=dt)
    u = [S.leray(I.cylindrical_shear_flow(N, seed=62, member=m, rho=0.05), 1.0) for m in range(M)]
    for m, x in enumerate(u):
        p.set_initial(m, x)
    p.step(nsteps)
    g = p.ensemble_stats(N)
    uT = np.stack([S.integrate(x, prm, nsteps)[0] for x in u])
    ref = T.ensemble_stats(uT, 1.0, prm)
    for key in ("mean", "var"):
        a, b = np.asarray(g[key])[0], ref[key][0]
        assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(b)), key
    for m in range(M):
        assert abs(p.get_state(m).cpu().numpy()[0, 0, 0, 0] - u[m][0, 0, 0, 0]) < 1e-15
    assert np.max(np.asarray(g["var"])[0]) > 0      # the samples differ
    p.close()


def test_physical_field_and_mesh_refinement_measures(lib):
    """Mesh refinement of the perturbed Taylor-Green ensemble (section 6.1) at
    small scale: the same 6 samples at 16^3 and 32^3 (FP64), fields from
    ns3d_physical_field (checked against the oracle), compared on the coarse
    grid points: sample, mean and variance differences and the 1-point
    Wasserstein distance of the u_x marginals (package = oracle definition;
    W1 >= the mean difference pointwise)."""
    from paper_2401_09843_gb300 import binding as B
    from paper_2401_09843_gb300.ensemble import wasserstein1_one_point
    M, dt, n = 6, 2e-4, 5
    prm = S.Params(L=1.0, eps0=1.0, nu=1e-3, dt_fixed=dt)
    fields = {}
    for N in (16, 32):
        u = [S.leray(I.perturbed_taylor_green(N, seed=601, member=m), 1.0) for m in range(M)]
        p = B.Plan([N] * M, B.NS3D_F64, L=1.0, eps0=1.0, nu=1e-3, dt_fixed=dt)
        for m, x in enumerate(u):
            p.set_initial(m, x)
        p.step(n)
        f = np.stack([p.physical_field(m).cpu().numpy() for m in range(M)])
        ref = T.physical_on_grid(S.integrate(u[0], prm, n)[0])
        assert np.max(np.abs(f[0] - ref)) < 1e-11 * np.max(np.abs(ref))
        fields[N] = f[:, 0]
        p.close()
    coarse, fine = fields[16], fields[32][:, ::2, ::2, ::2]
    w = wasserstein1_one_point(coarse, fine)
    assert abs(w - T.wasserstein1_one_point(coarse, fine)) < 1e-12
    mean_err = np.mean(np.abs(coarse.mean(axis=0) - fine.mean(axis=0)))
    var_err = np.mean(np.abs(coarse.var(axis=0, ddof=1) - fine.var(axis=0, ddof=1)))
    sample_err = np.mean(np.abs(coarse - fine))
    assert mean_err - 1e-15 <= w <= sample_err + 1e-15
    assert 0 < w < 0.1 and var_err >= 0


def _shell(k2):
    K = np.floor(np.sqrt(k2.astype(np.float64))).astype(np.int64)
    K += ((2 * K + 1) ** 2 <= 4 * k2)
    K -= (K > 0) & ((2 * K - 1) ** 2 > 4 * k2)
    return K


@pytest.mark.parametrize("N", [48, 128])
def test_spectra_are_compensated_and_reproducible(lib, N):
    """Each spectrum bin is the exactly rounded sum of its modes within a few
    ulps (compensated sums; a plain sum of ~10^5 terms drifts further), and two
    calls agree bit for bit (a fixed merge order, no atomics)."""
    import math
    from paper_2401_09843_gb300 import binding as B
    p = B.Plan([N], B.NS3D_F64, eps0=1.0)
    p.set_initial(0, I.random_spectrum(N, seed=77, k0=0.3 * N))
    a, b = p.ensemble_stats(N), p.ensemble_stats(N)
    for k in ("spectrum", "enstrophy_spectrum", "s2", "s2_ball"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    for k in ("energy", "enstrophy", "dissipation"):
        assert a[k] == b[k], k
    u = p.get_state(0).cpu().numpy()[..., : N // 2]       # drop the zero Nyquist kz plane
    p.close()
    e = np.sum(u.real ** 2 + u.imag ** 2, axis=0)
    e[..., 1:] *= 2.0                                     # mirror modes -k
    k = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + np.arange(N // 2)[None, None, :] ** 2
    K = _shell(k2).ravel()
    order = np.argsort(K, kind="stable")
    bounds = np.searchsorted(K[order], np.arange(N + 1))
    ev, zv = (0.5 * e).ravel()[order], (0.5 * k2 * e).ravel()[order]
    spec = np.array([math.fsum(ev[bounds[i]:bounds[i + 1]]) for i in range(N)])
    zspec = np.array([math.fsum(zv[bounds[i]:bounds[i + 1]]) for i in range(N)])
    tol = 8 * np.finfo(np.float64).eps                    # per-mode rounding + the merge
    assert np.all(np.abs(np.asarray(a["spectrum"]) - spec) <= tol * spec)
    assert np.all(np.abs(np.asarray(a["enstrophy_spectrum"]) - zspec) <= tol * zspec)
    assert abs(a["energy"] - math.fsum(ev)) <= tol * math.fsum(ev)
    assert abs(a["enstrophy"] - math.fsum(zv)) <= tol * math.fsum(zv)


@pytest.mark.parametrize("Ma,Mb", [(6, 6), (5, 7)])
def test_mesh_refinement_measures_on_the_gpu(lib, Ma, Mb):
    """ns3d_mesh_refinement between a 16^3 and a 32^3 level of one plan
    (perturbed Taylor-Green samples of section 6.1, FP64, a few steps) against
    the oracle's definitions on the oracle's own fields: the 1-point
    Wasserstein distance (integral of |F_a - F_b| per point), the mean,
    variance and (equal counts) paired sample errors and the MC error bar,
    per component, averaged over the coarse points."""
    from paper_2401_09843_gb300 import binding as B
    dt, n = 2e-4, 4
    prm = S.Params(L=1.0, eps0=1.0, nu=1e-3, dt_fixed=dt)
    Ns = [16] * Ma + [32] * Mb
    u0 = [S.leray(I.perturbed_taylor_green(N, seed=611, member=m if m < Ma else m - Ma), 1.0)
          for m, N in enumerate(Ns)]
    p = B.Plan(Ns, B.NS3D_F64, L=1.0, eps0=1.0, nu=1e-3, dt_fixed=dt)
    for m, x in enumerate(u0):
        p.set_initial(m, x)
    p.step(n)
    got = p.mesh_refinement(16, 32)
    p.close()
    f = [T.physical_on_grid(S.integrate(x, prm, n)[0]) for x in u0]
    a = np.stack(f[:Ma])                                  # (Ma, 3, 16, 16, 16)
    b = np.stack(f[Ma:])[:, :, ::2, ::2, ::2]             # fine values at the coarse points
    assert got["coarse_members"] == Ma and got["fine_members"] == Mb
    for c in range(3):
        w = T.wasserstein1_one_point(a[:, c], b[:, c])
        assert abs(got["w1"][c] - w) < 1e-10 * w + 1e-15, (c, got["w1"][c], w)
        me = np.mean(np.abs(a[:, c].mean(0) - b[:, c].mean(0)))
        va, vb = a[:, c].var(0, ddof=1), b[:, c].var(0, ddof=1)
        ve = np.mean(np.abs(va - vb))
        se = np.mean(np.sqrt(va / Ma + vb / Mb))
        assert abs(got["mean_err"][c] - me) < 1e-10 * me + 1e-15
        assert abs(got["var_err"][c] - ve) < 1e-9 * ve + 1e-15
        assert abs(got["mc_se"][c] - se) < 1e-10 * se
        if Ma == Mb:
            sp = np.mean(np.abs(a[:, c] - b[:, c]))
            assert abs(got["sample_err"][c] - sp) < 1e-10 * sp
            assert got["mean_err"][c] <= got["w1"][c] + 1e-15 <= sp + 2e-15
        else:
            assert got["sample_err"][c] == -1.0
        assert got["w1"][c] > 0
