"""Pins for the oracle's statistics (Parseval, brute-force structure function,
zero variance, Chan merge) and for its discrete adjoint (dot-product tests,
central finite differences, the Beltrami closed form)."""
import math

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import adjoint as A
from oracle import solver as S
from oracle import stats as T

TWO_PI = 2 * math.pi


# --------------------------------------------------------------------------- statistics

def test_spectrum_sums_to_energy():
    uh = I.random_spectrum(16, seed=3, k0=3.0)
    assert abs(T.energy_spectrum(uh).sum() - S.energy(uh)) < 1e-15
    tg = T.energy_spectrum(I.taylor_green(16))
    assert abs(tg[2] - 0.125) < 1e-15 and abs(tg.sum() - 0.125) < 1e-15   # round(sqrt 3) = 2


@pytest.mark.parametrize("N,L", [(8, TWO_PI), (16, TWO_PI), (12, 1.0)])
def test_structure_function_spectral_equals_brute_force(N, L):
    uh = I.random_spectrum(N, seed=N, k0=2.0)
    u = T.physical_on_grid(uh)
    assert np.allclose(T.structure_function_spectral(uh, L), T.structure_function_brute(u),
                       rtol=1e-12, atol=1e-15)


def test_ball_mean_cos_against_quadrature():
    """j(q) = average of cos(kappa . h) over the ball |h| <= r, by Gauss-Legendre
    quadrature in spherical coordinates with kappa off the axes."""
    xr, wr = np.polynomial.legendre.leggauss(40)
    xt, wt = np.polynomial.legendre.leggauss(40)
    nphi = 96
    phi = 2 * np.pi * np.arange(nphi) / nphi
    rho = 0.5 * (xr + 1.0)                           # r = 1, rho in (0, 1)
    mu = xt                                          # cos(theta)
    R, MU, PH = np.meshgrid(rho, mu, phi, indexing="ij")
    W = (0.5 * wr)[:, None, None] * wt[None, :, None] * (2 * np.pi / nphi)
    st = np.sqrt(1.0 - MU ** 2)
    h = np.stack([R * st * np.cos(PH), R * st * np.sin(PH), R * MU])
    d = np.array([1.0, -2.0, 2.0]) / 3.0
    for q in (0.05, 0.7, 1.0, 2.5, 7.0):
        kap = q * d
        f = np.cos(np.tensordot(kap, h, axes=1)) * R ** 2
        avg = np.sum(W * f) / (4.0 * np.pi / 3.0)
        assert abs((1.0 - avg) - T.one_minus_ball_mean_cos(q)) < 1e-13 * max(1.0, 1.0 - avg), q
    # both branches meet at q = 1
    a = T.one_minus_ball_mean_cos(np.nextafter(1.0, 0.0))
    b = T.one_minus_ball_mean_cos(1.0)
    assert abs(a - b) < 1e-15


def test_ball_structure_function_pins():
    L = 2 * math.pi
    N = 16
    u = I.random_spectrum(N, seed=9, k0=3.0)
    # small r: 2 (1 - j(q)) ~ q^2 / 5, so S2_ball(r) / r^2 -> (1/5) sum |kappa|^2 |u_hat|^2 = 2 Z / 5
    Z = float(np.sum(T.enstrophy_spectrum(u, L)))
    r = 1e-4
    assert abs(T.structure_function_ball(u, L, r)[0] / r ** 2 - 0.4 * Z) < 1e-6 * Z
    # large r: j -> 0, S2_ball -> 2 sum |u_hat|^2 = 4 E for a field without mean flow
    E = float(np.sum(T.energy_spectrum(u)))
    assert abs(T.structure_function_ball(u, L, 1e8)[0] - 4 * E) < 1e-12 * E
    # one mode u = (0, sin 3x, 0): |sin 3(x + h_x) - sin 3x|^2 averages over x to
    # 1 - cos 3 h_x, and over the ball to 1 - j(3 r)
    one = np.zeros((3, N, N, N // 2 + 1), complex)
    one[1, 3, 0, 0] = -0.5j
    one[1, N - 3, 0, 0] = 0.5j
    rs = np.arange(1, N // 2 + 1) * L / N
    got = T.structure_function_ball(one, L)
    j = 3 * (np.sin(3 * rs) - 3 * rs * np.cos(3 * rs)) / (3 * rs) ** 3
    assert np.max(np.abs(got - (1.0 - j))) < 1e-14


def test_identical_samples_have_zero_variance_and_exact_moments():
    uh = I.random_spectrum(8, seed=1)
    st = T.ensemble_stats(np.stack([uh] * 4), TWO_PI)
    u = T.physical_on_grid(uh)
    assert np.max(np.abs(st["var"])) < 1e-28
    assert np.max(np.abs(st["spectrum_stderr"])) < 1e-15
    assert np.allclose(st["mean"], u, atol=1e-15)
    assert np.allclose(st["second"][1], u[0] * u[1], atol=1e-15)


def test_chan_merge_equals_two_pass():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((37, 5)) * 3 + 1
    a = T.welford(x[:20])
    b = T.welford(x[20:])
    n, m, q = T.chan_merge(a, b)
    assert n == 37
    assert np.allclose(m, x.mean(0), rtol=1e-14)
    assert np.allclose(q / (n - 1), x.var(0, ddof=1), rtol=1e-13)


def test_mean_and_stderr_of_known_samples():
    s = np.array([[1.0], [3.0], [5.0]])
    m, se = T.mean_and_stderr(s)
    assert m[0] == 3.0 and abs(se[0] - math.sqrt(4.0 / 3.0)) < 1e-15


# --------------------------------------------------------------------------- adjoint

def _rand_field(N, seed, div_free=True):
    if div_free:
        return I.random_spectrum(N, seed=seed, k0=2.5, energy=0.3)
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((3, N, N, N))
    return I.coefficients_of(u)


@pytest.mark.parametrize("div_free", [True, False])
def test_adjoint_rhs_dot_product(div_free):
    N = 12
    prm = S.Params(nu=0.01, eps0=1.0)
    u = I.random_spectrum(N, seed=1, k0=2.5)
    du = _rand_field(N, 2, div_free)
    w = _rand_field(N, 3, div_free)
    lhs = S.inner(w, A.tangent_rhs(u, du, prm))
    rhs = S.inner(A.adjoint_rhs(u, w, prm), du)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_tangent_rhs_matches_finite_difference():
    N = 12
    prm = S.Params(nu=0.01, eps0=1.0)
    u = I.random_spectrum(N, seed=1, k0=2.5)
    du = _rand_field(N, 2)
    h = 1e-5
    fd = (S.rhs(u + h * du, prm) - S.rhs(u - h * du, prm)) / (2 * h)
    tl = A.tangent_rhs(u, du, prm)
    assert np.linalg.norm((fd - tl).ravel()) < 1e-9 * np.linalg.norm(tl.ravel())


def test_rk3_adjoint_step_dot_product():
    N = 12
    prm = S.Params(nu=0.01, eps0=1.0)
    u = I.random_spectrum(N, seed=5, k0=2.5)
    du = _rand_field(N, 6, False)
    lam = _rand_field(N, 7, False)
    dt = 0.05
    lhs = S.inner(lam, A.rk3_tangent_step(u, du, dt, prm))
    rhs = S.inner(A.rk3_adjoint_step(u, lam, dt, prm), du)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_band_energy_gradient_finite_differences():
    N = 12
    prm = S.Params(nu=0.01, eps0=1.0)
    dt, n = 0.05, 4
    u0 = I.random_spectrum(N, seed=8, k0=2.5)
    g = A.grad_band_energy(u0, prm, n, dt, 2.0, 4.0, checkpoint_every=3)

    def J(u):
        un, _, _ = S.integrate(u, prm.with_(dt_fixed=dt), n)
        return A.band_energy(un, 2.0, 4.0)

    for seed in (1, 2):
        v = I.random_spectrum(N, seed=100 + seed, k0=2.5, energy=0.5)
        h = 1e-4
        fd = (J(u0 + h * v) - J(u0 - h * v)) / (2 * h)
        assert abs(fd - S.inner(g, v)) < 2e-8 * abs(fd)


def test_checkpointing_does_not_change_gradient():
    N = 8
    prm = S.Params(nu=0.01, eps0=1.0)
    u0 = I.random_spectrum(N, seed=2, k0=2.0)
    g1 = A.grad_band_energy(u0, prm, 5, 0.05, 1.0, 3.0, checkpoint_every=0)
    g2 = A.grad_band_energy(u0, prm, 5, 0.05, 1.0, 3.0, checkpoint_every=2)
    assert np.array_equal(g1, g2)


def test_beltrami_gradient_closed_form():
    """For a Beltrami field on the shell |k| = K the nonlinear term and its
    adjoint act only through gradients: the divergence-free part of dJ/du0 is
    r(-lambda_K dt)^(2n) u0 when K is in the band, 0 otherwise."""
    N = 16
    prm = S.Params(nu=0.05, s=1.5, theta=0.25, eps0=2.0)
    u0 = I.single_shell_beltrami(N, K=3)
    lamK = 0.05 * 9 + 2.0 / 256.0 * 27.0 * (1.0 - (4.0 / 9.0) ** 4)
    dt, n = 0.05, 3
    r = 1 - lamK * dt + (lamK * dt) ** 2 / 2 - (lamK * dt) ** 3 / 6
    g = A.grad_band_energy(u0, prm, n, dt, 2.5, 3.5)
    pg = S.leray(g, TWO_PI)
    assert np.linalg.norm((pg - r ** (2 * n) * u0).ravel()) < 1e-13 * np.linalg.norm(u0.ravel())
    g_out = A.grad_band_energy(u0, prm, n, dt, 4.0, 6.0)
    assert np.max(np.abs(S.leray(g_out, TWO_PI))) < 1e-15


def test_enstrophy_spectrum_pins():
    """Beltrami field at shell K (omega = K u): Z(K) = K^2 E(K), zero on other
    shells; a random divergence-free field: Z(K) = 1/2 sum |kappa|^2 |u|^2 by
    shell (|kappa x u|^2 = |kappa|^2 |u|^2 when kappa . u = 0)."""
    N, K = 16, 3
    u = I.beltrami_abc(N, K=K)
    E, Z = T.energy_spectrum(u), T.enstrophy_spectrum(u, S.TWO_PI)
    assert abs(Z[K] - K * K * E[K]) < 1e-13 * Z[K]
    assert np.sum(np.abs(np.delete(Z, K))) < 1e-13 * Z[K]
    v = I.random_spectrum(N, seed=3, k0=3.0)
    kx, ky, kz = S.wavenumbers(N)
    k2 = (kx * kx + ky * ky + kz * kz).astype(float)
    e = 0.5 * np.sum(np.abs(v) ** 2, axis=0) * S.half_weights(N) * k2
    ref = np.bincount(np.broadcast_to(T.shell_index(N), e.shape).ravel(), weights=e.ravel(),
                      minlength=N)[:N]
    assert np.allclose(T.enstrophy_spectrum(v, S.TWO_PI), ref, rtol=1e-13, atol=1e-15)


def test_dissipation_rate_is_minus_dE_dt():
    """D = sum lambda_k |u_k|^2 equals -Re<u, R(u)> (the nonlinear term
    conserves energy under exact dealiasing)."""
    N = 16
    prm = S.Params(nu=0.02, eps0=1.0)
    u = I.random_spectrum(N, seed=8, k0=3.0)
    D = T.dissipation_rate(u, prm)
    assert abs(D + S.inner(u, S.rhs(u, prm))) < 1e-12 * D


def test_vorticity_magnitude_taylor_green():
    """u = (sin x cos y cos z, -cos x sin y cos z, 0): omega = (-cos x sin y sin z,
    -sin x cos y sin z, 2 sin x sin y cos z) by hand."""
    N = 16
    x = np.arange(N) * 2 * np.pi / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    w2 = ((np.cos(X) * np.sin(Y) * np.sin(Z)) ** 2 + (np.sin(X) * np.cos(Y) * np.sin(Z)) ** 2
          + (2 * np.sin(X) * np.sin(Y) * np.cos(Z)) ** 2)
    got = T.vorticity_magnitude(I.taylor_green(N), S.TWO_PI)
    assert np.max(np.abs(got - np.sqrt(w2))) < 1e-13


def test_cylindrical_shear_flow_initial_data():
    """rho = 0, delta = 0: u_x is -1 inside the unperturbed cylinder r <= 1/4
    and 1 outside, so its mean is 1 - 2 (pi/16) up to the grid sampling of the
    disc; the perturbed data are seeded per member and stay x-dependent."""
    N = 64
    u = I.cylindrical_shear_flow(N, seed=1, rho=0.0, delta=0.0)
    # the k = 0 coefficient is the grid mean of the sampled step (the Nyquist
    # modes the retained set drops do not touch it)
    assert abs(u[0, 0, 0, 0].real - (1 - 2 * np.pi / 16)) < 0.02 and abs(u[0, 0, 0, 0].imag) < 1e-15
    ux = S.to_physical(u, N)[0]
    assert np.mean(np.abs(np.abs(ux) - 1.0) < 0.05) > 0.8     # away from the interface (Gibbs)
    assert np.max(np.abs(u[1:])) < 1e-15
    v0 = I.cylindrical_shear_flow(32, seed=1, member=0)
    v1 = I.cylindrical_shear_flow(32, seed=1, member=1)
    assert np.linalg.norm(v0 - v1) > 1e-3 * np.linalg.norm(v0)
    assert np.array_equal(v0, I.cylindrical_shear_flow(32, seed=1, member=0))
    # smooth profile: about +-1 (the truncation to the retained modes overshoots a little),
    # with the x dependence of the displaced axis
    w = S.to_physical(I.cylindrical_shear_flow(32, seed=2, rho=0.1), 32)[0]
    assert np.max(np.abs(w)) < 1.2 and np.std(w.mean(axis=(1, 2))) > 1e-4


def test_wasserstein_pins():
    """W1 closed forms: Dirac masses |a - b|; a shift by c gives |c|;
    (delta_0 + delta_1)/2 against delta_1/2 gives 1/2; W1 >= |mean difference|;
    equal counts: the mean distance of the sorted samples."""
    rng = np.random.default_rng(4)
    assert abs(T.wasserstein1_1d([0.3], [1.7]) - 1.4) < 1e-15
    x = rng.standard_normal(50)
    assert abs(T.wasserstein1_1d(x, x + 0.25) - 0.25) < 1e-12
    assert abs(T.wasserstein1_1d([0.0, 1.0], [0.5]) - 0.5) < 1e-15
    a, b = rng.standard_normal(40), 0.5 + 2 * rng.standard_normal(25)
    assert T.wasserstein1_1d(a, b) >= abs(a.mean() - b.mean()) - 1e-12
    c = rng.standard_normal(40)
    assert abs(T.wasserstein1_1d(a, c) - np.mean(np.abs(np.sort(a) - np.sort(c)))) < 1e-12


def test_package_wasserstein_matches_oracle():
    from paper_2401_09843_gb300.ensemble import wasserstein1_one_point
    rng = np.random.default_rng(5)
    a, b, c = rng.standard_normal((8, 3, 4)), rng.standard_normal((8, 3, 4)), rng.standard_normal((5, 3, 4))
    assert abs(wasserstein1_one_point(a, b) - T.wasserstein1_one_point(a, b)) < 1e-12
    assert abs(wasserstein1_one_point(a, c) - T.wasserstein1_one_point(a, c)) < 1e-12
