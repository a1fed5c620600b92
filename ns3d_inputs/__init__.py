"""Seeded synthetic initial data for the 3D periodic incompressible solver.

This module is shared by the CPU oracle, the tests and the benchmark.  It
produces Fourier coefficients of initial velocity fields; it contains none of
the solver's arithmetic (no transforms of the method, no projection operator,
no right-hand side).  The only transform used is numpy's own ``rfftn`` to turn
a formula sampled on the grid (or white noise) into coefficients.

Layout of every field returned here (the "D1" layout of the library
boundary): complex128 array of shape ``(3, N, N, N//2 + 1)``, index
``[component][kx][ky][kz]``, with integer wavenumber k = i for i < N/2 and
k = i - N otherwise along x and y, and kz = 0..N/2 along z.  The coefficient
normalisation is

    u_hat[k] = N^-3 * sum_x u(x) exp(-i kappa.x),   kappa = (2 pi / L) k,

so that u(x) = sum_k u_hat[k] exp(i kappa.x) over the full (Hermitian)
spectrum.  Modes outside the retained set |k_i| <= N/2 - 1 (the Nyquist
planes kx = N/2, ky = N/2, kz = N/2) are always zero: this is the projection
P_N applied to the initial data (eq. shv_disc, u(0) = P_N u0).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "wavenumbers",
    "truncate",
    "taylor_green",
    "taylor_green_2d",
    "beltrami_abc",
    "single_shell_beltrami",
    "random_spectrum",
    "perturbed_taylor_green",
    "coefficients_of",
]


def wavenumbers(N: int):
    """Integer wavenumbers (kx, ky, kz) broadcastable to the D1 array shape."""
    k = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    kx = k[:, None, None]
    ky = k[None, :, None]
    kz = np.arange(N // 2 + 1, dtype=np.int64)[None, None, :]
    return kx, ky, kz


def retained_mask(N: int) -> np.ndarray:
    """Boolean mask of the retained modes |k_i| <= N/2 - 1 on the D1 grid."""
    kx, ky, kz = wavenumbers(N)
    h = N // 2
    return (np.abs(kx) < h) & (np.abs(ky) < h) & (kz < h)


def truncate(uhat: np.ndarray) -> np.ndarray:
    """Zero every mode outside the retained set (drop the Nyquist planes)."""
    N = uhat.shape[-2]
    out = np.array(uhat, dtype=np.complex128, copy=True)
    out *= retained_mask(N)
    return out


def coefficients_of(u: np.ndarray) -> np.ndarray:
    """Fourier coefficients (D1 layout, N^-3 normalisation) of a real field
    sampled on the N^3 grid x_j = j L / N, shape (3, N, N, N)."""
    N = u.shape[-1]
    return truncate(np.fft.rfftn(u, axes=(1, 2, 3)) / float(N) ** 3)


def _grid(N: int, L: float):
    x = np.arange(N) * (L / N)
    return np.meshgrid(x, x, x, indexing="ij")


def taylor_green(N: int, L: float = 2 * np.pi) -> np.ndarray:
    """3D Taylor-Green vortex u = (sin x cos y cos z, -cos x sin y cos z, 0)
    with x scaled by 2 pi / L (so the field is one period of the domain)."""
    X, Y, Z = _grid(N, L)
    a = 2 * np.pi / L
    u = np.stack([
        np.sin(a * X) * np.cos(a * Y) * np.cos(a * Z),
        -np.cos(a * X) * np.sin(a * Y) * np.cos(a * Z),
        np.zeros_like(X),
    ])
    return coefficients_of(u)


def taylor_green_2d(N: int, L: float = 2 * np.pi, axis_free: int = 2) -> np.ndarray:
    """2D Taylor-Green vortex embedded in 3D, constant along ``axis_free``:
    u = (sin x cos y, -cos x sin y, 0) for axis_free = 2.  It is a steady
    solution of the Euler equations (the nonlinear term is a gradient)."""
    X, Y, Z = _grid(N, L)
    a = 2 * np.pi / L
    g = [X, Y, Z]
    free = axis_free
    p, q = [i for i in range(3) if i != free]
    u = np.zeros((3, N, N, N))
    u[p] = np.sin(a * g[p]) * np.cos(a * g[q])
    u[q] = -np.cos(a * g[p]) * np.sin(a * g[q])
    return coefficients_of(u)


def beltrami_abc(N: int, K: int = 1, A: float = 1.0, B: float = 0.7,
                 C: float = 0.4, L: float = 2 * np.pi) -> np.ndarray:
    """Arnold-Beltrami-Childress field at wavenumber K:
    u = (A sin Kz + C cos Ky, B sin Kx + A cos Kz, C sin Ky + B cos Kx).
    curl u = K u, so (u . grad) u = grad(|u|^2 / 2): the nonlinear term is a
    pure gradient and the Leray projection removes it."""
    X, Y, Z = _grid(N, L)
    a = 2 * np.pi / L * K
    u = np.stack([
        A * np.sin(a * Z) + C * np.cos(a * Y),
        B * np.sin(a * X) + A * np.cos(a * Z),
        C * np.sin(a * Y) + B * np.cos(a * X),
    ])
    return coefficients_of(u)


def single_shell_beltrami(N: int, seed: int = 7, K: int = 3, L: float = 2 * np.pi) -> np.ndarray:
    """A random Beltrami field on one integer shell |k|^2 = K^2 built from
    the modes of the three coordinate axes with random amplitudes/phases.
    Every mode satisfies i k x u_k = |k| u_k, so curl u = |k| u and the
    nonlinear term projects out exactly."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 11])))
    uhat = np.zeros((3, N, N, N // 2 + 1), dtype=np.complex128)
    for d in range(3):
        # helical vector h with i k x h = |k| h for k = K e_d:
        # h = e_a + i e_b with (d, a, b) a cyclic permutation of (0, 1, 2).
        a, b = (d + 1) % 3, (d + 2) % 3
        h = np.zeros(3, dtype=np.complex128)
        h[a] = 1.0
        h[b] = 1j
        v = complex(rng.standard_normal(), rng.standard_normal()) * h
        if d == 2:
            uhat[:, 0, 0, K] += v          # the mirror -k is implied by storage
        else:
            ip = [0, 0]
            ip[d] = K
            im = [0, 0]
            im[d] = (-K) % N
            uhat[:, ip[0], ip[1], 0] += v  # kz = 0 plane holds both k and -k
            uhat[:, im[0], im[1], 0] += np.conj(v)
    return truncate(uhat)


def random_spectrum(N: int, seed: int, member: int = 0, k0: float = 4.0,
                    energy: float = 0.5, L: float = 2 * np.pi) -> np.ndarray:
    """Seeded random divergence-free field with energy spectrum
    E(k) proportional to k^4 exp(-2 (k/k0)^2), total energy
    E = 1/2 sum_k |u_hat_k|^2 = ``energy`` over the full spectrum.

    Recipe: i.i.d. N(0,1) white noise g(x) per component on the N^3 grid,
    drawn from numpy's Philox generator keyed by (seed, member); g_hat its
    coefficients; u_hat_k = a(|k|) (i k x g_hat_k) / |k| for the retained
    k != 0 with a(k) = sqrt(E(k) / (4 pi k^2)), then one global factor that
    fixes the energy.  i k x g is the curl of a random vector potential: it
    is divergence-free and keeps the Hermitian symmetry of a real field.
    """
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(member)])))
    g = rng.standard_normal((3, N, N, N))
    ghat = np.fft.rfftn(g, axes=(1, 2, 3)) / float(N) ** 3
    kx, ky, kz = wavenumbers(N)
    kv = [np.broadcast_to(kx, ghat.shape[1:]), np.broadcast_to(ky, ghat.shape[1:]),
          np.broadcast_to(kz, ghat.shape[1:])]
    kmag = np.sqrt(kv[0] ** 2.0 + kv[1] ** 2.0 + kv[2] ** 2.0)
    safe = np.where(kmag > 0, kmag, 1.0)
    spec = safe ** 4 * np.exp(-2.0 * (safe / k0) ** 2)
    amp = np.sqrt(spec / (4 * np.pi * safe ** 2)) / safe
    curl = np.stack([
        1j * (kv[1] * ghat[2] - kv[2] * ghat[1]),
        1j * (kv[2] * ghat[0] - kv[0] * ghat[2]),
        1j * (kv[0] * ghat[1] - kv[1] * ghat[0]),
    ])
    uhat = truncate(curl * amp * (kmag > 0))
    e = _energy_d1(uhat)
    if e > 0:
        uhat *= np.sqrt(energy / e)
    return uhat


def perturbed_taylor_green(N: int, seed: int, member: int = 0,
                           delta: float = 0.025) -> np.ndarray:
    """Perturbed Taylor-Green initial measure on the unit torus (L = 1):
    the base flow (cos 2pi x sin 2pi y sin 2pi z, -sin 2pi x cos 2pi y sin 2pi z, 0)
    plus, per component d, (1/8) sum over (i,j,k) in {0,1}^3 of
    delta_{d,i,j,k} a_i(4 pi x) a_j(4 pi y) a_k(4 pi z) with a_0 = sin,
    a_1 = cos and delta ~ U[-0.025, 0.025] (section 6.1 of the paper)."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(member), 61])))
    X, Y, Z = _grid(N, 1.0)
    tp = 2 * np.pi
    u = np.stack([
        np.cos(tp * X) * np.sin(tp * Y) * np.sin(tp * Z),
        -np.sin(tp * X) * np.cos(tp * Y) * np.sin(tp * Z),
        np.zeros_like(X),
    ])
    alpha = (np.sin, np.cos)
    d = rng.uniform(-delta, delta, size=(3, 2, 2, 2))
    for c in range(3):
        for i in range(2):
            for j in range(2):
                for k in range(2):
                    u[c] += d[c, i, j, k] / 8.0 * alpha[i](2 * tp * X) * alpha[j](2 * tp * Y) * alpha[k](2 * tp * Z)
    return coefficients_of(u)


def cylindrical_shear_flow(N: int, seed: int, member: int = 0, rho: float = 0.05,
                           delta: float = 0.025, p: int = 10) -> np.ndarray:
    """Cylindrical shear flow initial measure on the unit torus (L = 1), the
    paper's section 6.2: u = tanh(2 pi (r - 0.25) / rho) (rho = 0: -1 for
    r <= 0.25, else 1), v = w = 0, with
    r^2 = (y - 0.5 + s_y(x))^2 + (z - 0.5 + s_z(x))^2 and
    s_d(x) = delta sum_{k=1..p} a_k^d sin(2 pi k x - b_k^d), a ~ U[0, 1],
    b ~ U[0, 2 pi] independent per sample and direction."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(member), 67])))
    a = rng.uniform(0.0, 1.0, size=(2, p))
    b = rng.uniform(0.0, 2 * np.pi, size=(2, p))
    X, Y, Z = _grid(N, 1.0)
    k = np.arange(1, p + 1)
    sig = [delta * np.sum(a[d][:, None, None, None] *
                          np.sin(2 * np.pi * k[:, None, None, None] * X[None] - b[d][:, None, None, None]),
                          axis=0) for d in range(2)]
    r = np.sqrt((Y - 0.5 + sig[0]) ** 2 + (Z - 0.5 + sig[1]) ** 2)
    if rho > 0:
        ux = np.tanh(2 * np.pi * (r - 0.25) / rho)
    else:
        ux = np.where(r <= 0.25, -1.0, 1.0)
    return coefficients_of(np.stack([ux, np.zeros_like(ux), np.zeros_like(ux)]))


def _energy_d1(uhat: np.ndarray) -> float:
    """1/2 sum over the full spectrum of |u_hat|^2 from D1 half storage."""
    w = np.full(uhat.shape[-1], 2.0)
    w[0] = 1.0
    N = uhat.shape[-2]
    if N % 2 == 0:
        w[-1] = 1.0
    return 0.5 * float(np.sum(np.abs(uhat) ** 2 * w))


def sparse_random(N: int, seed: int, nmodes: int = 40, kmax: int = 0, energy: float = 0.5) -> np.ndarray:
    """A real divergence-free field with ``nmodes`` random retained modes
    (|k_i| < kmax, default N/2), each i k x g / |k| for a Gaussian g, scaled
    to the given energy.  Sparse spectra let the Galerkin product be summed
    mode pair by mode pair at any N."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), 97])))
    h = N // 2
    kmax = kmax or h
    uhat = np.zeros((3, N, N, h + 1), dtype=np.complex128)
    for _ in range(nmodes):
        k = rng.integers(-(kmax - 1), kmax, size=3)
        k[2] = abs(k[2])
        if not k.any():
            continue
        g = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        v = 1j * np.cross(k, g) / np.linalg.norm(k)
        ix, iy = int(k[0]) % N, int(k[1]) % N
        if k[2] == 0:   # keep the kz = 0 plane Hermitian
            uhat[:, ix, iy, 0] += v
            uhat[:, (-int(k[0])) % N, (-int(k[1])) % N, 0] += np.conj(v)
        else:
            uhat[:, ix, iy, int(k[2])] += v
    uhat = truncate(uhat)
    e = _energy_d1(uhat)
    return uhat * np.sqrt(energy / e) if e > 0 else uhat


def sparse_modes(N: int, seed: int, nmodes: int = 40, kmax: int = 0, energy: float = 0.5):
    """A real divergence-free field given by its nonzero modes, for grids too
    large to hold densely on the host: returns (K, V), K (n, 3) integer wave
    vectors as stored in the D1 layout (k_z >= 0; on the k_z = 0 plane both k
    and -k are listed, with conjugate coefficients) and V (n, 3) complex128
    coefficients.  Modes are i k x g / |k| for Gaussian g with |k_i| < kmax
    (default N/2), scaled to the given energy 1/2 sum over the full spectrum."""
    rng = np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), 101])))
    h = N // 2
    kmax = kmax or h
    acc = {}
    for _ in range(nmodes):
        k = rng.integers(-(kmax - 1), kmax, size=3)
        k[2] = abs(k[2])
        if not k.any():
            continue
        g = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        v = 1j * np.cross(k, g) / np.linalg.norm(k)
        key = (int(k[0]), int(k[1]), int(k[2]))
        acc[key] = acc.get(key, 0) + v
        if k[2] == 0:
            mk = (-key[0], -key[1], 0)
            acc[mk] = acc.get(mk, 0) + np.conj(v)
    K = np.array(sorted(acc), dtype=np.int64).reshape(-1, 3)
    V = np.array([acc[tuple(k)] for k in K.tolist()], dtype=np.complex128).reshape(-1, 3)
    w = np.where(K[:, 2] > 0, 2.0, 1.0)
    e = 0.5 * float(np.sum(w * np.sum(np.abs(V) ** 2, axis=1)))
    return K, (V * np.sqrt(energy / e) if e > 0 else V)


def modes_of(uhat: np.ndarray, rtol: float = 0.0):
    """(K, V) of the entries of a D1 array above rtol times its largest (K
    signed, k_z >= 0); rtol > 0 drops the round-off of a sampled field."""
    N = uhat.shape[-2]
    mag = np.max(np.abs(uhat), axis=0)
    nz = np.nonzero(mag > rtol * np.max(mag)) if rtol > 0 else np.nonzero(np.any(uhat != 0, axis=0))
    kx = np.where(nz[0] < N // 2, nz[0], nz[0] - N)
    ky = np.where(nz[1] < N // 2, nz[1], nz[1] - N)
    K = np.stack([kx, ky, nz[2]], axis=1).astype(np.int64)
    return K, uhat[:, nz[0], nz[1], nz[2]].T.copy()
