"""Ensemble statistics of an approximate statistical solution (oracle).

TEST INFRASTRUCTURE ONLY.

Algorithm 1 (section 2.1) approximates the statistical solution by the
empirical measure (1/M) sum_i delta_{u_i(t)} of M Monte Carlo samples; the
writers of section 2.4 reduce it to observables.  The paper prints no
formulas for them; the definitions used (both here and in the library) are:

* mean field            m_i(x)    = (1/M) sum_m u_{m,i}(x)        on the N^3 grid
* second moments        E[u_i u_j](x) = (1/M) sum_m u_{m,i} u_{m,j}  (i <= j,
                        order 00 01 02 11 12 22)
* pointwise variance    v_i(x)    = (1/(M-1)) sum_m (u_{m,i} - m_i)^2
* energy spectrum       E(K)      = 1/2 sum_{k : round(|k|) = K} |u_hat_k|^2
                        (full spectrum, K = 0 .. N-1), mean over samples
* structure function    S2(r)     = (1/3) sum_d <|u(x + r e_d) - u(x)|^2>_x
                                  = (1/3) sum_d sum_k 2 |u_hat_k|^2 (1 - cos(kappa_d r)),
                        r = j L / N, j = 1 .. N/2
* ball-averaged S2      S2_ball(r) = < (1/|B_r|) int_{|h|<=r} |u(x+h) - u(x)|^2 dh >_x
                                  = sum_k 2 |u_hat_k|^2 (1 - 3 (sin q - q cos q) / q^3),
                        q = |kappa| r, at the same r
* enstrophy spectrum    Z(K)      = 1/2 sum_{k : round(|k|) = K} |omega_hat_k|^2,
                        omega_hat = i kappa x u_hat (the vorticity the paper's
                        section 6.1 shows, as a spectrum writer)
* dissipation rate      D         = sum_k lambda_k |u_hat_k|^2 (full spectrum):
                        -dE/dt of the spectral equation (section 2.3), whose
                        dealiased nonlinear term conserves energy
* vorticity magnitude   |omega(x)| on the N^3 grid
* 1-point Wasserstein distance between two ensembles (the paper's section 6.1
  mesh-refinement measure): at each grid point the samples define empirical
  one-point marginals mu_x, nu_x; W1(mu_x, nu_x) = integral |F_mu - F_nu| dt
  (1D), and the distance is its mean over the points
* Monte Carlo standard error of a sample mean: sqrt(var / M).

Sample sets are merged with the pairwise formula of Chan, Golub and LeVeque
(count, mean, sum of squared deviations).
"""
from __future__ import annotations

import math

import numpy as np

from .solver import curl, dissipation, half_weights, to_physical, wavenumbers

PAIRS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def physical_on_grid(uhat: np.ndarray) -> np.ndarray:
    """u at the N^3 grid points (no padding)."""
    return to_physical(uhat, uhat.shape[-2])


def shell_index(N: int) -> np.ndarray:
    """round(|k|) on the D1 grid, as int."""
    kx, ky, kz = wavenumbers(N)
    k2 = (kx * kx + ky * ky + kz * kz).astype(np.float64)
    return np.floor(np.sqrt(k2) + 0.5).astype(np.int64)


def energy_spectrum(uhat: np.ndarray) -> np.ndarray:
    N = uhat.shape[-2]
    e = 0.5 * np.sum(np.abs(uhat) ** 2, axis=0) * half_weights(N)
    sh = np.broadcast_to(shell_index(N), e.shape)
    return np.bincount(sh.ravel(), weights=e.ravel(), minlength=N)[:N]


def structure_function_spectral(uhat: np.ndarray, L: float) -> np.ndarray:
    N = uhat.shape[-2]
    kx, ky, kz = wavenumbers(N)
    e = np.sum(np.abs(uhat) ** 2, axis=0) * half_weights(N)
    out = np.zeros(N // 2)
    for j in range(1, N // 2 + 1):
        r = j * L / N
        acc = 0.0
        for kd in (kx, ky, kz):
            kap = (2 * math.pi / L) * kd
            acc += np.sum(e * 2.0 * (1.0 - np.cos(kap * r)))
        out[j - 1] = acc / 3.0
    return out


def one_minus_ball_mean_cos(q):
    """1 - j(q), j(q) = (1/|B_r|) int_{|h| <= r} cos(kappa . h) dh = 3 (sin q - q cos q) / q^3
    with q = |kappa| r (the ball's indicator in Fourier space; j(0) = 1).

    For q < 1 the difference is summed from the Taylor series of
    sin q - q cos q = sum_{n >= 1} (-1)^(n+1) 2n q^(2n+1) / (2n+1)!, which gives
    1 - j(q) = sum_{n >= 2} (-1)^n 6n q^(2n-2) / (2n+1)!  (the direct formula
    cancels there); 14 terms leave less than 1e-28."""
    q = np.asarray(q, dtype=np.float64)
    small = q < 1.0
    qs = np.where(small, q, 0.0)
    series = np.zeros_like(q)
    for n in range(2, 16):
        series += (-1) ** n * 6 * n / math.factorial(2 * n + 1) * qs ** (2 * n - 2)
    ql = np.where(small, 1.0, q)
    direct = 1.0 - 3.0 * (np.sin(ql) - ql * np.cos(ql)) / ql ** 3
    return np.where(small, series, direct)


def structure_function_ball(uhat: np.ndarray, L: float, r=None) -> np.ndarray:
    """Ball-averaged second-order structure function
        S2_ball(r) = < (1/|B_r|) int_{|h| <= r} |u(x + h) - u(x)|^2 dh >_x
                   = sum_k |u_hat_k|^2 2 (1 - j(|kappa| r))          (full spectrum),
    by default at r = j L / N, j = 1 .. N/2.  The axis-lag S2 above averages the
    increment over the three axis directions instead of the ball."""
    N = uhat.shape[-2]
    kx, ky, kz = wavenumbers(N)
    kap = (2 * math.pi / L) * np.sqrt((kx ** 2 + ky ** 2 + kz ** 2).astype(np.float64))
    e = np.sum(np.abs(uhat) ** 2, axis=0) * half_weights(N)
    rs = np.arange(1, N // 2 + 1) * L / N if r is None else np.atleast_1d(np.asarray(r, float))
    return np.array([np.sum(e * 2.0 * one_minus_ball_mean_cos(kap * rr)) for rr in rs])


def structure_function_brute(u: np.ndarray) -> np.ndarray:
    """S2 from grid values by shifting whole grid points (r = j L / N)."""
    N = u.shape[-1]
    out = np.zeros(N // 2)
    for j in range(1, N // 2 + 1):
        acc = 0.0
        for ax in (1, 2, 3):
            acc += np.mean(np.sum((np.roll(u, -j, axis=ax) - u) ** 2, axis=0))
        out[j - 1] = acc / 3.0
    return out


def enstrophy_spectrum(uhat: np.ndarray, L: float) -> np.ndarray:
    """Z(K) = 1/2 sum over round(|k|) = K of |omega_hat_k|^2, full spectrum;
    the vorticity from its definition omega_hat = i kappa x u_hat."""
    return energy_spectrum(curl(uhat, L))


def dissipation_rate(uhat: np.ndarray, prm) -> float:
    """D = sum_k lambda_k |u_hat_k|^2 over the full spectrum."""
    N = uhat.shape[-2]
    w = half_weights(N)
    return float(np.sum(w * dissipation(N, prm) * np.sum(np.abs(uhat) ** 2, axis=0)))


def vorticity_magnitude(uhat: np.ndarray, L: float) -> np.ndarray:
    """|omega(x)| at the N^3 grid points."""
    w = physical_on_grid(curl(uhat, L))
    return np.sqrt(np.sum(w * w, axis=0))


def mean_and_stderr(samples: np.ndarray):
    """Sample mean and Monte Carlo standard error along axis 0."""
    M = samples.shape[0]
    mean = samples.mean(axis=0)
    if M < 2:
        return mean, np.zeros_like(mean)
    var = samples.var(axis=0, ddof=1)
    return mean, np.sqrt(var / M)


def ensemble_stats(uhats: np.ndarray, L: float, prm=None) -> dict:
    """All writer statistics of an ensemble given as (M, 3, N, N, N/2+1);
    the dissipation rate needs the solver parameters prm."""
    M = uhats.shape[0]
    N = uhats.shape[-2]
    phys = np.stack([physical_on_grid(u) for u in uhats])           # (M,3,N,N,N)
    mean = phys.mean(axis=0)
    second = np.stack([(phys[:, i] * phys[:, j]).mean(axis=0) for i, j in PAIRS])
    var = phys.var(axis=0, ddof=1) if M > 1 else np.zeros_like(mean)
    spec = np.stack([energy_spectrum(u) for u in uhats])
    s2 = np.stack([structure_function_spectral(u, L) for u in uhats])
    en = spec.sum(axis=1)
    spec_m, spec_se = mean_and_stderr(spec)
    s2_m, s2_se = mean_and_stderr(s2)
    s2b_m, s2b_se = mean_and_stderr(np.stack([structure_function_ball(u, L) for u in uhats]))
    en_m, en_se = mean_and_stderr(en)
    zspec = np.stack([enstrophy_spectrum(u, L) for u in uhats])
    zs_m, zs_se = mean_and_stderr(zspec)
    z_m, z_se = mean_and_stderr(zspec.sum(axis=1))
    out = dict(M=M, N=N, mean=mean, second=second, var=var,
               spectrum=spec_m, spectrum_stderr=spec_se,
               s2=s2_m, s2_stderr=s2_se, s2_ball=s2b_m, s2_ball_stderr=s2b_se,
               energy=float(en_m), energy_stderr=float(en_se),
               enstrophy_spectrum=zs_m, enstrophy_spectrum_stderr=zs_se,
               enstrophy=float(z_m), enstrophy_stderr=float(z_se))
    if prm is not None:
        d_m, d_se = mean_and_stderr(np.array([dissipation_rate(u, prm) for u in uhats]))
        out.update(dissipation=float(d_m), dissipation_stderr=float(d_se))
    return out


def chan_merge(a, b):
    """Merge two (count, mean, M2) triples; M2 = sum of squared deviations."""
    na, ma, qa = a
    nb, mb, qb = b
    n = na + nb
    if n == 0:
        return (0, ma, qa)
    d = mb - ma
    return (n, ma + d * (nb / n), qa + qb + d * d * (na * nb / n))


def welford(samples: np.ndarray):
    """(count, mean, M2) of samples along axis 0, one sample at a time."""
    n, mean, m2 = 0, np.zeros_like(samples[0], dtype=np.float64), np.zeros_like(samples[0], dtype=np.float64)
    for x in samples:
        n += 1
        d = x - mean
        mean = mean + d / n
        m2 = m2 + d * (x - mean)
    return n, mean, m2


def wasserstein1_1d(a: np.ndarray, b: np.ndarray) -> float:
    """W1 between the empirical measures of the 1D samples a and b, from its
    definition as the integral of |F_a(t) - F_b(t)| over t: both empirical
    CDFs are constant between consecutive points of the merged samples."""
    a = np.sort(np.asarray(a, dtype=np.float64).ravel())
    b = np.sort(np.asarray(b, dtype=np.float64).ravel())
    t = np.sort(np.concatenate([a, b]))
    total = 0.0
    for lo, hi in zip(t[:-1], t[1:]):
        if hi > lo:
            Fa = np.searchsorted(a, lo, side="right") / len(a)
            Fb = np.searchsorted(b, lo, side="right") / len(b)
            total += abs(Fa - Fb) * (hi - lo)
    return total


def wasserstein1_one_point(sa: np.ndarray, sb: np.ndarray) -> float:
    """Mean over the points of W1 between the one-point marginals of two
    ensembles of fields, sa (Ma, ...) and sb (Mb, ...) on the same points."""
    sa = np.asarray(sa).reshape(sa.shape[0], -1)
    sb = np.asarray(sb).reshape(sb.shape[0], -1)
    return float(np.mean([wasserstein1_1d(sa[:, i], sb[:, i]) for i in range(sa.shape[1])]))
