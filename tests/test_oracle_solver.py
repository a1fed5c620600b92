"""Pins for the oracle solver: closed forms, invariants, symmetries.

Every expected value here comes from the mathematics of the method (section
2.2-2.3 of the paper), not from the oracle itself:
* the Taylor-Green right-hand side worked out by hand (below),
* products of single Fourier modes (trigonometric identities),
* Beltrami fields, whose nonlinear term is a gradient,
* the SSP-RK3 stability polynomial for a linear decay,
* conservation of energy and helicity by the inviscid Galerkin system,
* divergence, Hermitian symmetry, translation and axis-permutation
  equivariance.
"""
import math

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

TWO_PI = 2 * math.pi
EULER = S.Params(nu=0.0, eps0=0.0)


def sample(f, N, L=TWO_PI):
    x = np.arange(N) * (L / N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return f(X, Y, Z)


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


# --------------------------------------------------------------------------- transforms

@pytest.mark.parametrize("N,P", [(8, 12), (16, 24), (16, 32)])
def test_taylor_green_physical_values(N, P):
    uh = I.taylor_green(N)
    u = S.to_physical(uh, P)
    ref = sample(lambda X, Y, Z: np.stack([np.sin(X) * np.cos(Y) * np.cos(Z),
                                           -np.cos(X) * np.sin(Y) * np.cos(Z),
                                           0 * X]), P)
    assert np.max(np.abs(u - ref)) < 1e-14
    assert abs(S.energy(uh) - 0.125) < 1e-15


def _single_mode(N, k):
    """Coefficients of cos(k . x) (modes +-k with 1/2)."""
    return I.coefficients_of(np.stack([sample(lambda X, Y, Z: np.cos(k[0] * X + k[1] * Y + k[2] * Z), N)] * 3))[0]


@pytest.mark.parametrize("P,exact", [(12, True), (13, True), (8, False)])
def test_product_of_two_modes(P, exact):
    """cos(a.x) cos(b.x) = 1/2 cos((a+b).x) + 1/2 cos((a-b).x); with N = 8 the
    mode a+b = (6,1,2) lies outside K_N and must be dropped, not aliased."""
    N = 8
    a, b = (3, 1, 0), (3, 0, 2)
    ua = S.to_physical(_single_mode(N, a)[None], P)[0]
    ub = S.to_physical(_single_mode(N, b)[None], P)[0]
    got = S.to_spectral((ua * ub)[None], N)[0]
    diff = np.array(a) - np.array(b)
    expect = 0.5 * I.coefficients_of(np.stack([sample(
        lambda X, Y, Z: np.cos(diff[0] * X + diff[1] * Y + diff[2] * Z), N)] * 3))[0]
    err = np.max(np.abs(got - expect))
    if exact:
        assert err < 1e-15
    else:
        assert err > 0.1          # P = N aliases (6,1,2) onto (-2,1,2)


# --------------------------------------------------------------------------- projection

def test_leray_projection_properties():
    rng = np.random.default_rng(0)
    N, L = 12, 3.0
    b = rng.standard_normal((3, N, N, N // 2 + 1)) + 1j * rng.standard_normal((3, N, N, N // 2 + 1))
    k = S.kappa(N, L)
    pb = S.leray(b, L)
    div = k[0] * pb[0] + k[1] * pb[1] + k[2] * pb[2]
    assert np.max(np.abs(div)) < 1e-13 * np.max(np.abs(b)) * np.max(np.abs(k[0]))
    assert np.max(np.abs(S.leray(pb, L) - pb)) < 1e-14 * np.max(np.abs(b))
    phi = rng.standard_normal((N, N, N // 2 + 1))
    grad = np.stack([1j * k[j] * phi for j in range(3)])
    assert np.max(np.abs(S.leray(grad, L))) < 1e-13 * np.max(np.abs(grad))
    assert np.all(pb[:, 0, 0, 0] == 0)


# --------------------------------------------------------------------------- nonlinear term

def test_taylor_green_rhs_closed_form():
    """For u = (sin x cos y cos z, -cos x sin y cos z, 0):
    (u.grad)u = 1/2 (sin 2x, sin 2y, 0) cos^2 z.  Its divergence-free part is
    -R = 1/8 (sin 2x cos 2z, sin 2y cos 2z, -(cos 2x + cos 2y) sin 2z), the
    remainder being the gradient of (cos 2x + cos 2y)(2 + cos 2z)/16."""
    N = 8
    uh = I.taylor_green(N)
    expect = I.coefficients_of(sample(lambda X, Y, Z: -0.125 * np.stack([
        np.sin(2 * X) * np.cos(2 * Z),
        np.sin(2 * Y) * np.cos(2 * Z),
        -(np.cos(2 * X) + np.cos(2 * Y)) * np.sin(2 * Z)]), N))
    for form in (0, 1, 2):
        R = S.rhs(uh, EULER, form=form)
        assert np.max(np.abs(R - expect)) < 1e-15, form


@pytest.mark.parametrize("field", ["abc1", "abc2", "shell", "tg2d"])
def test_beltrami_and_2d_tg_nonlinear_term_projects_out(field):
    N = 16
    uh = {"abc1": lambda: I.beltrami_abc(N, 1),
          "abc2": lambda: I.beltrami_abc(N, 2, 0.3, -1.1, 0.8),
          "shell": lambda: I.single_shell_beltrami(N, K=3),
          "tg2d": lambda: I.taylor_green_2d(N)}[field]()
    for form in (0, 1, 2):
        b, _ = S.nonlinear(uh, EULER, form=form)
        pb = S.leray(b, TWO_PI)
        assert np.max(np.abs(pb)) < 1e-14 * max(1.0, np.max(np.abs(b))), form


def test_2d_taylor_green_nonlinear_term_closed_forms():
    """b before the projection, each form against its own closed form for
    u = (sin x cos y, -cos x sin y, 0): (u.grad)u = 1/2 (sin 2x, sin 2y, 0) (and
    div(u u) is the same, u being divergence-free), so forms 0 and 1 give
    b = -1/2 (sin 2x, sin 2y, 0); with omega = (0, 0, 2 sin x sin y),
    u x omega = (-sin 2x sin^2 y, -sin^2 x sin 2y, 0) for form 2.  A transposed
    gradient (grad |u|^2/2 instead) or a swapped cross product fails."""
    N = 16
    uh = I.taylor_green_2d(N)
    adv = I.coefficients_of(sample(lambda X, Y, Z: -0.5 * np.stack([
        np.sin(2 * X), np.sin(2 * Y), 0.0 * Z]), N))
    rot = I.coefficients_of(sample(lambda X, Y, Z: np.stack([
        -np.sin(2 * X) * np.sin(Y) ** 2, -np.sin(X) ** 2 * np.sin(2 * Y), 0.0 * Z]), N))
    for form, expect in ((0, adv), (1, adv), (2, rot)):
        b, umax = S.nonlinear(uh, EULER, form=form)
        assert np.max(np.abs(b - expect)) < 1e-15, form
        assert abs(umax - 1.0) < 1e-15     # max |sin x cos y| + |cos x sin y| = 1 at x = y = pi/4


def test_three_nonlinear_forms_agree():
    N = 16
    uh = I.random_spectrum(N, seed=5, k0=3.0)
    r0 = S.rhs(uh, EULER, form=0)
    for form in (1, 2):
        assert rel(S.rhs(uh, EULER, form=form), r0) < 1e-13


# --------------------------------------------------------------------------- dissipation and RK3

def test_dissipation_values_by_hand():
    N = 16
    prm = S.Params(nu=0.01, s=1.5, theta=0.5, eps0=1.0, mN_coef=1.0)   # m_N = 4, eps_N = 1/256
    lam = S.dissipation(N, prm)
    # k = (1,0,0): |k| <= m_N, no hyper-viscosity
    assert abs(lam[1, 0, 0] - 0.01) < 1e-16
    # k = (4,0,0): |k| = m_N exactly, still undamped by Q
    assert abs(lam[4, 0, 0] - 0.16) < 1e-15
    # k = (3,3,0): |k|^2 = 18, Q = 1 - (16/18)^2
    q = 1.0 - (16.0 / 18.0) ** 2
    assert abs(lam[3, 3, 0] - (0.18 + 18.0 ** 1.5 * q / 256.0)) < 1e-14
    # k = (-5,2,6): |k|^2 = 65
    q = 1.0 - (16.0 / 65.0) ** 2
    assert abs(lam[N - 5, 2, 6] - (0.65 + 65.0 ** 1.5 * q / 256.0)) < 1e-13
    # step form of Q and domain length L = 1 (kappa = 2 pi k)
    prm1 = prm.with_(q_form=1, L=1.0)
    lam1 = S.dissipation(N, prm1)
    kap2 = (TWO_PI ** 2) * 18.0
    assert abs(lam1[3, 3, 0] - (0.01 * kap2 + kap2 ** 1.5 / 256.0)) < 1e-10


@pytest.mark.parametrize("field,K2", [("abc1", 1), ("abc2", 4), ("shell", 9)])
def test_rk3_beltrami_decay_is_stability_polynomial(field, K2):
    """Beltrami fields evolve linearly: u_n = r(-lambda_K dt)^n u_0 with
    r(z) = 1 + z + z^2/2 + z^3/6 (SSP-RK3 on u' = -lambda u)."""
    N = 16
    uh = {"abc1": lambda: I.beltrami_abc(N, 1),
          "abc2": lambda: I.beltrami_abc(N, 2, 0.3, -1.1, 0.8),
          "shell": lambda: I.single_shell_beltrami(N, K=3)}[field]()
    prm = S.Params(nu=0.05, s=1.5, theta=0.25, eps0=2.0)      # m_N = 2 -> |k|>2 damped
    mN2 = 2.0 ** 2
    epsN = 2.0 / 16.0 ** 2
    q = 0.0 if K2 <= mN2 else 1.0 - (mN2 / K2) ** 4
    lamK = 0.05 * K2 + epsN * K2 ** 1.5 * q
    dt, n = 0.07, 6
    u, t, _ = S.integrate(uh, prm.with_(dt_fixed=dt), n)
    r = 1 - lamK * dt + (lamK * dt) ** 2 / 2 - (lamK * dt) ** 3 / 6
    assert rel(u, uh * r ** n) < 1e-13
    assert abs(t - n * dt) < 1e-15


# --------------------------------------------------------------------------- invariants

def test_inviscid_energy_and_helicity_are_conserved_by_rhs():
    N = 16
    uh = I.random_spectrum(N, seed=9, k0=3.0) + 0.3 * I.single_shell_beltrami(N, K=2)
    R = S.rhs(uh, EULER)
    scale = math.sqrt(S.inner(uh, uh) * S.inner(R, R))
    assert abs(S.inner(uh, R)) < 1e-14 * scale
    w = S.curl(uh, TWO_PI)
    assert abs(S.inner(w, R)) < 1e-14 * math.sqrt(S.inner(w, w) * S.inner(R, R))


def test_energy_budget_with_dissipation():
    N = 16
    prm = S.Params(nu=0.02, s=1.5, theta=0.5, eps0=1.0)
    uh = I.random_spectrum(N, seed=9, k0=3.0)
    R = S.rhs(uh, prm)
    lam = S.dissipation(N, prm)
    dEdt = S.inner(uh, R)
    expect = -S.inner(uh, lam * uh)
    assert abs(dEdt - expect) < 1e-14 * abs(expect)


def test_taylor_green_initial_dissipation_rate():
    """All eight TG modes sit on |k|^2 = 3: dE/dt(0) = -2 lambda_3 E(0)."""
    N = 32
    prm = S.Params(nu=0.01, s=1.5, theta=0.5, eps0=1.0)       # m_N^2 = 32 > 3: no SV
    uh = I.taylor_green(N)
    dEdt = S.inner(uh, S.rhs(uh, prm))
    assert abs(dEdt - (-2 * 0.01 * 3 * 0.125)) < 1e-16


def test_constraints_after_steps():
    N = 16
    prm = S.Params(nu=0.0, eps0=1.0, dt_fixed=0.02)
    uh = I.random_spectrum(N, seed=1, k0=3.0)
    mean0 = uh[:, 0, 0, 0].copy()
    u, _, _ = S.integrate(uh, prm, 3)
    assert S.divergence_ratio(u, TWO_PI) < 1e-14
    p = u[:, :, :, 0]
    mirror = np.conj(p[:, (-np.arange(N)) % N][:, :, (-np.arange(N)) % N])
    assert np.max(np.abs(p - mirror)) < 1e-15
    assert np.all(u[:, 0, 0, 0] == mean0)
    assert np.all(u[:, N // 2] == 0) and np.all(u[:, :, N // 2] == 0) and np.all(u[..., N // 2] == 0)


def test_axis_permutation_equivariance():
    N = 12
    prm = S.Params(nu=0.01, eps0=1.0)
    uh = I.random_spectrum(N, seed=4, k0=2.5)
    R = S.rhs(uh, prm)
    # swap x <-> y: component 0 <-> 1 and axes kx <-> ky
    sw = lambda a: a[[1, 0, 2]].transpose(0, 2, 1, 3)
    assert rel(S.rhs(sw(uh), prm), sw(R)) < 1e-13


def test_translation_equivariance():
    """u(x + a) has coefficients u_hat_k exp(i kappa.a); the dealiased RHS
    commutes with any translation a (not only grid shifts)."""
    N = 12
    prm = S.Params(nu=0.01, eps0=1.0)
    uh = I.random_spectrum(N, seed=4, k0=2.5)
    k = S.kappa(N, TWO_PI)
    a = (0.3, -1.1, 2.2)
    ph = np.exp(1j * (k[0] * a[0] + k[1] * a[1] + k[2] * a[2]))
    assert rel(S.rhs(uh * ph, prm), S.rhs(uh, prm) * ph) < 1e-13


def test_two_dimensional_field_stays_two_dimensional():
    N = 16
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((N, N))
    X = sample(lambda X, Y, Z: X, N)[:, :, 0]
    # u = (d psi/dy, -d psi/dx, 0) built with numpy's spectral derivative
    ph = np.fft.fft2(psi)
    kk = np.fft.fftfreq(N, 1.0 / N)
    kx, ky = kk[:, None], kk[None, :]
    ph = ph * (np.abs(kx) < 5) * (np.abs(ky) < 5)
    ux = np.real(np.fft.ifft2(1j * ky * ph))
    uy = np.real(np.fft.ifft2(-1j * kx * ph))
    u = np.stack([np.repeat(ux[:, :, None], N, 2), np.repeat(uy[:, :, None], N, 2), np.zeros((N, N, N))])
    uh = I.coefficients_of(u)
    uh /= math.sqrt(S.energy(uh) / 0.5)
    out, _, _ = S.integrate(uh, S.Params(nu=0.01, eps0=1.0, dt_fixed=0.01), 4)
    assert np.max(np.abs(out[:, :, :, 1:])) < 1e-15
    assert np.max(np.abs(out[2])) < 1e-15


def test_cfl_time_step_and_clipping():
    N = 16
    prm = S.Params(cfl=0.5)
    uh = I.taylor_green(N)
    _, umax = S.rhs(uh, prm, return_umax=True)
    # max |sin x cos y cos z| + |cos x sin y cos z| = 1 on the padded grid (x = y = pi/4 -> 1)
    assert abs(umax - 1.0) < 1e-12
    _, dt = S.rk3_step(uh, prm)
    assert abs(dt - 0.5 * (TWO_PI / N)) < 1e-12
    _, dt2 = S.rk3_step(uh, prm, t=0.99, t_end=1.0)
    assert abs(dt2 - 0.01) < 1e-15
    u3, dt3 = S.rk3_step(uh, prm, t=1.0, t_end=1.0)
    assert dt3 == 0.0 and np.array_equal(u3, uh)


def test_padded_size_rule():
    assert S.padded_size(32) == 48 and S.padded_size(256) == 384 and S.padded_size(1024) == 1536
    assert S.padded_size(22) == 35          # 33 = 3*11 is not 7-smooth, 34 = 2*17 neither
    assert S.padded_size(10) == 15
    assert all(S.is_7_smooth(S.padded_size(n)) and S.padded_size(n) * 2 >= 3 * n for n in range(2, 200, 2))


@pytest.mark.parametrize("N", [12, 16, 24])
def test_rhs_sparse_matches_transform_rhs(N):
    """The mode-list Galerkin sum (used at grid sizes too large to hold) equals
    the padded-transform RHS on a dense grid, for a sparse field with modes up
    to the band edge."""
    K, V = I.sparse_modes(N, seed=N, nmodes=20)
    u = np.zeros((3, N, N, N // 2 + 1), complex)
    u[:, K[:, 0] % N, K[:, 1] % N, K[:, 2]] = V.T
    assert abs(S.energy(u) - 0.5) < 1e-14 and S.divergence_ratio(u, S.TWO_PI) < 1e-14
    prm = S.Params(nu=0.01, eps0=1.0)
    ref = S.rhs(u, prm)
    Ko, R = S.rhs_sparse(K, V, N, prm)
    got = np.zeros_like(ref)
    got[:, Ko[:, 0] % N, Ko[:, 1] % N, Ko[:, 2]] = R.T
    assert np.linalg.norm(got - ref) < 1e-14 * np.linalg.norm(ref)
    K2, V2 = I.modes_of(u)
    assert np.array_equal(np.sort(K2, axis=0), np.sort(K, axis=0))


@pytest.mark.parametrize("N", [12, 16, 24])
def test_rhs_by_convolution_matches_transform_rhs(N):
    """The Galerkin product summed over mode pairs of a dense D1 array (the
    sparse-spectrum check used on full-size grids) equals the padded-transform
    RHS; visiting the pairs in small row blocks changes no bit."""
    u = I.sparse_random(N, seed=3 * N, nmodes=12)
    prm = S.Params(nu=0.01, eps0=1.0)
    ref = S.rhs(u, prm)
    got = S.rhs_by_convolution(u, prm)
    assert np.linalg.norm(got - ref) < 1e-14 * np.linalg.norm(ref)
    b_one = S.nonlinear_by_convolution(u, prm)
    b_rows = S.nonlinear_by_convolution(u, prm, chunk_pairs=7)
    assert np.array_equal(b_one, b_rows)


@pytest.mark.parametrize("N", [16, 24])
def test_rk3_step_with_convolution_rhs_matches_transform_step(N):
    """One SSP-RK3 step composed from the mode-pair Galerkin sum (three stages,
    the support growing by pair sums at each) equals the padded-transform
    step; the increment u+ - u agrees too, so a wrong stage weight shows."""
    u = I.sparse_random(N, seed=5 * N, nmodes=4)
    prm = S.Params(nu=0.0, eps0=1.0, dt_fixed=0.01)
    ref, dt = S.rk3_step(u, prm)
    got, dt2 = S.rk3_step(u, prm, rhs_fn=lambda v: S.rhs_by_convolution(v, prm))
    assert dt == dt2 == 0.01
    assert np.linalg.norm(got - ref) < 1e-14 * np.linalg.norm(ref)
    assert np.linalg.norm((got - u) - (ref - u)) < 1e-13 * np.linalg.norm(ref - u)
    # the step reached modes far outside the initial support
    assert np.count_nonzero(np.any(ref != 0, axis=0)) > 20 * np.count_nonzero(np.any(u != 0, axis=0))
    with pytest.raises(ValueError):
        S.rk3_step(u, prm.with_(dt_fixed=0.0), rhs_fn=lambda v: S.rhs_by_convolution(v, prm))


def _square(x):
    return x * x


def test_process_pool_map_gives_identical_rhs():
    """The per-component transforms of one RHS run through a spawn-started
    process pool when one is installed: the result is bitwise that of the
    serial map."""
    import concurrent.futures as cf
    import multiprocessing as mp
    N = 16
    u = I.random_spectrum(N, seed=77)
    prm = S.Params(nu=0.01, eps0=1.0)
    serial = S.rhs(u, prm)
    with cf.ProcessPoolExecutor(2, mp_context=mp.get_context("spawn")) as ex:
        old = S.set_map(ex.map)
        try:
            par = S.rhs(u, prm)
        finally:
            S.set_map(old)
    assert np.array_equal(par, serial)
    assert S.set_map(None) is map
