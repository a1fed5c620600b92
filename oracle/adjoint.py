"""Discrete adjoint of the SSP-RK3 step (oracle).

TEST INFRASTRUCTURE ONLY.  The paper has no adjoint; this differentiates its
discretisation (the right-hand side of section 2.3 and eq. RK3) exactly
("discretise, then differentiate") in the real inner product
<a, b> = Re sum_k conj(a_k) b_k over the full spectrum (= the spatial mean of
a . b).

Tangent-linear right-hand side at u (dt fixed):
    J(u) du = P(kappa) (-i kappa . F[du (x) u + u (x) du]) - lambda du.
Its adjoint, with w' = P(kappa) w:
    J(u)^T w = T_N F[ sum_l u_l (d_l w'_j + d_j w'_l) ] - lambda w,
obtained by integrating -div(du (x) u + u (x) du) against w' by parts.  With
P >= 3N/2 every product here is alias-free, so the continuous integration by
parts is exact for the truncated fields and this is the exact transpose of
the discrete J.

Adjoint of one RK3 step u -> u+ (stages u, u1, u2; lam the adjoint of u+):
    a2 = 2/3 (lam + dt J(u2)^T lam)
    a1 = 1/4 (a2 + dt J(u1)^T a2)
    a  = 1/3 lam + 3/4 a2 + a1 + dt J(u)^T a1.
"""
from __future__ import annotations

import numpy as np

from .solver import (Params, dissipation, kappa, leray, padded_size, retained_mask,
                     rhs, to_physical, to_spectral, wavenumbers)


def tangent_rhs(uhat, du, prm: Params, P=None):
    N = uhat.shape[-2]
    P = P or padded_size(N, prm.n_pad)
    k = kappa(N, prm.L)
    u = to_physical(uhat, P)
    d = to_physical(du, P)
    b = []
    for j in range(3):
        acc = 0
        for l in range(3):
            acc = acc + k[l] * to_spectral(d[j] * u[l] + u[j] * d[l], N)
        b.append(-1j * acc)
    b = np.stack(b)
    return (leray(b, prm.L) - dissipation(N, prm) * du) * retained_mask(N)


def adjoint_rhs(uhat, w, prm: Params, P=None):
    N = uhat.shape[-2]
    P = P or padded_size(N, prm.n_pad)
    k = kappa(N, prm.L)
    wp = leray(w * retained_mask(N), prm.L)
    u = to_physical(uhat, P)
    c = np.zeros_like(u)
    for j in range(3):
        for l in range(3):
            s_jl = to_physical(1j * k[l] * wp[j] + 1j * k[j] * wp[l], P)
            c[j] += u[l] * s_jl
    return (to_spectral(c, N) - dissipation(N, prm) * w) * retained_mask(N)


def rk3_stages(uhat, dt, prm: Params, P=None):
    u1 = uhat + dt * rhs(uhat, prm, P)
    u2 = 0.75 * uhat + 0.25 * u1 + 0.25 * dt * rhs(u1, prm, P)
    return uhat, u1, u2


def rk3_adjoint_step(uhat_n, lam_np1, dt, prm: Params, P=None):
    """Adjoint of one RK3 step at the forward state u_n (stages recomputed)."""
    u0, u1, u2 = rk3_stages(uhat_n, dt, prm, P)
    a2 = (2.0 / 3.0) * (lam_np1 + dt * adjoint_rhs(u2, lam_np1, prm, P))
    a1 = 0.25 * (a2 + dt * adjoint_rhs(u1, a2, prm, P))
    return lam_np1 / 3.0 + 0.75 * a2 + a1 + dt * adjoint_rhs(u0, a1, prm, P)


def rk3_tangent_step(uhat_n, du, dt, prm: Params, P=None):
    """Linearised RK3 step (for dot-product tests)."""
    u0, u1, u2 = rk3_stages(uhat_n, dt, prm, P)
    d1 = du + dt * tangent_rhs(u0, du, prm, P)
    d2 = 0.75 * du + 0.25 * (d1 + dt * tangent_rhs(u1, d1, prm, P))
    return du / 3.0 + (2.0 / 3.0) * (d2 + dt * tangent_rhs(u2, d2, prm, P))


def band_mask(N: int, k_lo: float, k_hi: float) -> np.ndarray:
    kx, ky, kz = wavenumbers(N)
    km = np.sqrt((kx * kx + ky * ky + kz * kz).astype(np.float64))
    return ((km >= k_lo) & (km < k_hi) & retained_mask(N)).astype(np.float64)


def band_energy(uhat, k_lo, k_hi) -> float:
    """J = 1/2 sum over the full spectrum of |u_hat_k|^2 for k_lo <= |k| < k_hi."""
    from .solver import inner
    m = band_mask(uhat.shape[-2], k_lo, k_hi)
    return 0.5 * inner(uhat * m, uhat * m)


def grad_band_energy(uhat0, prm: Params, nsteps: int, dt: float, k_lo: float, k_hi: float,
                     checkpoint_every: int = 0, P=None):
    """Gradient of J(u(T)) with respect to u_hat(0), T = nsteps dt.

    Forward pass keeps every ``checkpoint_every``-th state (all states when 0);
    the backward pass recomputes the states of one segment from its
    checkpoint and runs the adjoint steps of that segment in reverse."""
    from .solver import rk3_step
    C = checkpoint_every if checkpoint_every > 0 else 1
    ckpt = {0: np.array(uhat0, copy=True)}
    u = np.array(uhat0, copy=True)
    for n in range(nsteps):
        u, _ = rk3_step(u, prm, dt=dt, P=P)
        if (n + 1) % C == 0 and n + 1 < nsteps:
            ckpt[n + 1] = u.copy()
    lam = u * band_mask(u.shape[-2], k_lo, k_hi)
    starts = sorted(ckpt)
    for s in reversed(starts):
        end = min(s + C, nsteps)
        states = [ckpt[s]]
        for n in range(s, end - 1):
            nxt, _ = rk3_step(states[-1], prm, dt=dt, P=P)
            states.append(nxt)
        for n in range(end - 1, s - 1, -1):
            lam = rk3_adjoint_step(states[n - s], lam, dt, prm, P)
    return lam
