"""Plain FP64 restatement of the spectral hyper-viscosity solver (oracle).

TEST INFRASTRUCTURE ONLY: used by tests, smoke() and the CPU baseline.

Everything works on spectral fields in the "D1" layout: complex128 arrays of
shape (3, N, N, N//2 + 1), index [component][kx][ky][kz], wavenumbers
k = i (i < N/2) or i - N along x and y and kz = 0..N/2, coefficients
u_hat_k = N^-3 sum_x u(x) exp(-i kappa.x) with kappa = (2 pi / L) k.

What is computed, with the passage each step follows
----------------------------------------------------
* Retained set K_N = {k : |k_i| <= N/2 - 1}: the projection P_N of
  eq. shv_disc (section 2.2).  The paper's "|k|_inf <= N" is read as the modes
  of an N^3 grid with the Nyquist index dropped, so K_N = -K_N.
* Time derivative (section 2.3, the Fourier-space equation after eq. shv_disc):
      R(u_hat)_k = (I - kappa kappa^T / |kappa|^2) b_hat_k - lambda_k u_hat_k,
      b_hat_k = -i kappa^T . F[u (x) u]_k,   R_0 = 0,
  with the dissipation of eq. shv_disc read as damping (the printed "+" on
  eps_N |grad|^{2s} would amplify):
      lambda_k = nu |kappa|^2 + eps_N |kappa|^{2s} Q_k,
      Q_k = 0 for |k| <= m_N, else 1 - (m_N / |k|)^{(2s-1)/theta}  (q_form 0,
            the lower bound the paper requires) or 1 (q_form 1),
      eps_N = eps0 N^{1-2s},  m_N = mN_coef N^theta  (section 2.2 scalings).
* Algorithm 2 done the plain way: the whole spectrum is zero-padded to a P^3
  grid with P >= 3N/2 (section 3.1 padding rule), transformed back, the six
  products u_j u_l formed, transformed forward, and only K_N kept ("remove
  the upper third").  Not Algorithm 3: no axis-by-axis padding here.
* Two further nonlinear forms that the projection makes identical for a
  divergence-free field: advective (u . grad) u and rotational u x omega.
* SSP-RK3 (section 2.3, eq. RK3).
* CFL time step: dt = cfl (L / N) / max_x sum_i |u_i(x)| over the padded grid
  of the stage-1 field (the paper gives no formula; reading documented).
"""
from __future__ import annotations

from dataclasses import dataclass, replace
import math

import numpy as np

from . import fft as _fft

TWO_PI = 2.0 * math.pi

# The per-component transforms of one right-hand side are independent; they
# run through _MAP, the builtin map unless ``set_map`` installs a process
# pool's map.  Each component's arithmetic is the same either way, so the
# results are bitwise identical.
_MAP = map


def set_map(fn=None):
    """Install ``fn`` (e.g. a spawn-started process pool's ``map``) for the
    independent per-component transforms of ``nonlinear``; None restores the
    builtin map.  Returns the previous one."""
    global _MAP
    old = _MAP
    _MAP = map if fn is None else fn
    return old


@dataclass(frozen=True)
class Params:
    """Solver parameters (mirrors the library's ns3d_params)."""
    L: float = TWO_PI
    nu: float = 0.0
    s: float = 1.5
    theta: float = 0.5
    eps0: float = 1.0
    mN_coef: float = 1.0
    q_form: int = 0
    n_pad: int = 0
    nonlinear_form: int = 0
    cfl: float = 0.5
    dt_fixed: float = 0.0

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


# ---------------------------------------------------------------- grids

def is_7_smooth(n: int) -> bool:
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def padded_size(N: int, n_pad: int = 0) -> int:
    """P = n_pad if given, else the smallest 2^a 3^b 5^c 7^d >= 3N/2
    (section 3.1: any padded size >= 3N/2 keeps the product alias-free)."""
    if n_pad:
        return int(n_pad)
    P = (3 * N + 1) // 2
    while not is_7_smooth(P):
        P += 1
    return P


def wavenumbers(N: int):
    """Integer wavenumbers (kx, ky, kz) broadcastable to (N, N, N//2+1)."""
    k = np.fft.fftfreq(N, 1.0 / N).astype(np.int64)
    return (k[:, None, None], k[None, :, None],
            np.arange(N // 2 + 1, dtype=np.int64)[None, None, :])


def retained_mask(N: int) -> np.ndarray:
    kx, ky, kz = wavenumbers(N)
    h = N // 2
    return (np.abs(kx) < h) & (np.abs(ky) < h) & (kz < h)


def kappa(N: int, L: float):
    """Physical wavevector components kappa = (2 pi / L) k, full arrays."""
    kx, ky, kz = wavenumbers(N)
    a = TWO_PI / L
    shape = (N, N, N // 2 + 1)
    return [np.broadcast_to(a * kx, shape).astype(np.float64),
            np.broadcast_to(a * ky, shape).astype(np.float64),
            np.broadcast_to(a * kz, shape).astype(np.float64)]


def half_weights(N: int) -> np.ndarray:
    """Multiplicity of each stored kz column in the full spectrum: 1 for
    kz = 0 and kz = N/2, 2 otherwise."""
    w = np.full(N // 2 + 1, 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    return w[None, None, :]


def inner(a: np.ndarray, b: np.ndarray) -> float:
    """Real inner product over the full spectrum, Re sum_k conj(a_k) b_k,
    which equals the spatial mean of a(x) . b(x) (Parseval)."""
    N = a.shape[-2]
    return float(np.sum((np.conj(a) * b).real * half_weights(N)))


def energy(uhat: np.ndarray) -> float:
    """E = 1/2 <|u|^2> = 1/2 sum_k |u_hat_k|^2."""
    return 0.5 * inner(uhat, uhat)


def curl(uhat: np.ndarray, L: float) -> np.ndarray:
    """Spectral curl i kappa x u_hat."""
    k = kappa(uhat.shape[-2], L)
    return np.stack([
        1j * (k[1] * uhat[2] - k[2] * uhat[1]),
        1j * (k[2] * uhat[0] - k[0] * uhat[2]),
        1j * (k[0] * uhat[1] - k[1] * uhat[0]),
    ])


def helicity(uhat: np.ndarray, L: float) -> float:
    """H = <u . omega>."""
    return inner(uhat, curl(uhat, L))


def divergence_ratio(uhat: np.ndarray, L: float) -> float:
    """max |kappa . u_hat_k| / max |kappa| |u_hat_k| (0 for a div-free field)."""
    k = kappa(uhat.shape[-2], L)
    div = np.abs(k[0] * uhat[0] + k[1] * uhat[1] + k[2] * uhat[2])
    kk = np.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2)
    den = np.max(kk * np.sqrt(np.sum(np.abs(uhat) ** 2, axis=0)))
    return float(np.max(div) / den) if den > 0 else 0.0


# ---------------------------------------------------------------- dissipation

def damped_threshold(N: int, prm: Params) -> int:
    """Largest integer |k|^2 that is left undamped: |k| <= m_N  <=>  |k|^2 <= m_N^2."""
    mN2 = prm.mN_coef ** 2 * float(N) ** (2.0 * prm.theta)
    return int(math.floor(mN2 * (1.0 + 1e-12)))


def dissipation(N: int, prm: Params) -> np.ndarray:
    """lambda_k = nu |kappa|^2 + eps_N |kappa|^{2s} Q_k on the D1 grid."""
    kx, ky, kz = wavenumbers(N)
    return dissipation_of_k2((kx * kx + ky * ky + kz * kz).astype(np.float64), N, prm)


def dissipation_of_k2(k2: np.ndarray, N: int, prm: Params) -> np.ndarray:
    """lambda_k as a function of the integer |k|^2 (eq. shv_disc constants)."""
    k2 = np.asarray(k2, dtype=np.float64)
    a2 = (TWO_PI / prm.L) ** 2
    kap2 = a2 * k2
    eps_N = prm.eps0 * float(N) ** (1.0 - 2.0 * prm.s)
    mN2 = prm.mN_coef ** 2 * float(N) ** (2.0 * prm.theta)
    thr = damped_threshold(N, prm)
    safe = np.where(k2 > 0, k2, 1.0)
    if prm.q_form == 0:
        q = 1.0 - (mN2 / safe) ** ((2.0 * prm.s - 1.0) / (2.0 * prm.theta))
    else:
        q = np.ones_like(safe)
    q = np.where(k2 <= thr, 0.0, q)
    return prm.nu * kap2 + eps_N * kap2 ** prm.s * q


def max_dissipation(N: int, prm: Params) -> float:
    lam = dissipation(N, prm) * retained_mask(N)
    return float(np.max(lam))


# ---------------------------------------------------------------- padded transforms

def to_physical(uhat: np.ndarray, P: int) -> np.ndarray:
    """Values of the trigonometric polynomial sum_k u_hat_k exp(i kappa.x) at
    the P^3 grid points x_j = j L / P, for each leading component.

    The stored half spectrum is placed on a zero P^3 array, the modes with
    kz > 0 are mirrored to -k as conj(u_hat_k), and the real part of the
    unnormalised inverse DFT is returned (the real part takes the Hermitian
    part of the kz = 0 plane)."""
    lead = uhat.shape[:-3]
    N = uhat.shape[-2]
    assert P >= N
    kx, ky, kz = wavenumbers(N)
    m = np.broadcast_to(retained_mask(N), (N, N, N // 2 + 1))
    ix = np.broadcast_to(kx % P, m.shape)[m]
    iy = np.broadcast_to(ky % P, m.shape)[m]
    iz = np.broadcast_to(kz, m.shape)[m]
    Z = np.zeros(lead + (P, P, P), dtype=np.complex128)
    vals = uhat[..., m]
    Z[..., ix, iy, iz] = vals
    pos = iz > 0
    Z[..., (-ix[pos]) % P, (-iy[pos]) % P, (-iz[pos]) % P] = np.conj(vals[..., pos])
    return _fft.fftn(Z, axes=(-3, -2, -1), sign=+1).real


def to_spectral(b: np.ndarray, N: int) -> np.ndarray:
    """Coefficients P^-3 sum_j b(x_j) exp(-i kappa.x_j) of real grid data of
    size P^3, kept on the retained set K_N (D1 layout, other modes zero)."""
    P = b.shape[-1]
    full = _fft.fftn(b, axes=(-3, -2, -1), sign=-1) / float(P) ** 3
    kx, ky, kz = wavenumbers(N)
    shape = (N, N, N // 2 + 1)
    ix = np.broadcast_to(kx % P, shape)
    iy = np.broadcast_to(ky % P, shape)
    iz = np.broadcast_to(kz % P, shape)
    out = full[..., ix, iy, iz]
    return out * retained_mask(N)


def _to_physical_task(args):
    uh, P = args
    return to_physical(uh, P)


def _to_spectral_task(args):
    b, N = args
    return to_spectral(b, N)


# ---------------------------------------------------------------- right-hand side

def leray(b: np.ndarray, L: float) -> np.ndarray:
    """(I - kappa kappa^T / |kappa|^2) b, and 0 at k = 0."""
    N = b.shape[-2]
    k = kappa(N, L)
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    safe = np.where(k2 > 0, k2, 1.0)
    kb = (k[0] * b[0] + k[1] * b[1] + k[2] * b[2]) / safe
    out = np.stack([b[j] - k[j] * kb for j in range(3)])
    return out * (k2 > 0)


def nonlinear(uhat: np.ndarray, prm: Params, P: int | None = None, form: int | None = None):
    """b_hat (before projection) and max_x sum_i |u_i| on the padded grid.

    form 0 (divergence, the paper's): b_hat_j = -i sum_l kappa_l F[u_j u_l]
    form 1 (advective): b_hat = -F[(u . grad) u]
    form 2 (rotational): b_hat = F[u x omega]   (differs by a gradient)
    """
    N = uhat.shape[-2]
    P = P or padded_size(N, prm.n_pad)
    form = prm.nonlinear_form if form is None else form
    k = kappa(N, prm.L)
    u = np.stack(list(_MAP(_to_physical_task, [(uhat[c], P) for c in range(3)])))
    umax = float(np.max(np.abs(u[0]) + np.abs(u[1]) + np.abs(u[2])))
    if form == 0:
        pairs = [(j, l) for j in range(3) for l in range(j, 3)]
        Bhat = {}
        for (j, l), v in zip(pairs, _MAP(_to_spectral_task, [(u[j] * u[l], N) for j, l in pairs])):
            Bhat[j, l] = v
            Bhat[l, j] = v
        b = np.stack([-1j * sum(k[l] * Bhat[j, l] for l in range(3)) for j in range(3)])
    elif form == 1:
        a = np.zeros_like(u)
        for l in range(3):
            dl = to_physical(1j * k[l] * uhat, P)   # d/dx_l of every component
            for j in range(3):
                a[j] += u[l] * dl[j]
        b = -to_spectral(a, N)
    elif form == 2:
        w = to_physical(curl(uhat, prm.L), P)
        c = np.stack([u[1] * w[2] - u[2] * w[1],
                      u[2] * w[0] - u[0] * w[2],
                      u[0] * w[1] - u[1] * w[0]])
        b = to_spectral(c, N)
    else:
        raise ValueError("unknown nonlinear form")
    return b, umax


def rhs(uhat: np.ndarray, prm: Params, P: int | None = None, form: int | None = None,
        return_umax: bool = False):
    """R(u_hat) = Leray(b_hat) - lambda u_hat on K_N (zero elsewhere)."""
    N = uhat.shape[-2]
    b, umax = nonlinear(uhat, prm, P, form)
    R = leray(b, prm.L) - dissipation(N, prm) * uhat
    R = R * retained_mask(N)
    return (R, umax) if return_umax else R


# ---------------------------------------------------------------- time stepping

def cfl_dt(umax: float, N: int, prm: Params) -> float:
    return prm.cfl * (prm.L / N) / umax


def rk3_step(uhat: np.ndarray, prm: Params, dt: float | None = None, P: int | None = None,
             t: float = 0.0, t_end: float = 0.0, rhs_fn=None):
    """One SSP-RK3 step (eq. RK3):
        u1 = u + dt R(u)
        u2 = 3/4 u + 1/4 u1 + 1/4 dt R(u1)
        u+ = 1/3 u + 2/3 u2 + 2/3 dt R(u2)
    dt: given, else prm.dt_fixed if > 0, else the CFL step of the stage-1
    field; clipped so that t + dt <= t_end when t_end > 0 (a member that has
    reached t_end does not move).  rhs_fn: another evaluation of R (e.g.
    ``rhs_by_convolution`` for sparse spectra on large grids); it gives no
    CFL maximum, so dt or prm.dt_fixed must then be set.  Returns (u+, dt)."""
    N = uhat.shape[-2]
    if rhs_fn is None:
        R0, umax = rhs(uhat, prm, P, return_umax=True)
    else:
        R0, umax = rhs_fn(uhat), None
        if dt is None and not prm.dt_fixed > 0:
            raise ValueError("rhs_fn needs a given dt or prm.dt_fixed")
    if dt is None:
        dt = prm.dt_fixed if prm.dt_fixed > 0 else cfl_dt(umax, N, prm)
        if t_end > 0:
            dt = min(dt, t_end - t)
            if dt <= 0:
                return uhat.copy(), 0.0
    f = (lambda v: rhs(v, prm, P)) if rhs_fn is None else rhs_fn
    u1 = uhat + dt * R0
    u2 = 0.75 * uhat + 0.25 * u1 + 0.25 * dt * f(u1)
    un = uhat / 3.0 + (2.0 / 3.0) * u2 + (2.0 / 3.0) * dt * f(u2)
    return un, dt


def integrate(uhat: np.ndarray, prm: Params, nsteps: int, P: int | None = None,
              t0: float = 0.0, t_end: float = 0.0, dts=None):
    """nsteps RK3 steps; returns (u, t, list of dt)."""
    u = np.array(uhat, copy=True)
    t = t0
    used = []
    for n in range(nsteps):
        dt_n = None if dts is None else dts[n]
        u, dt = rk3_step(u, prm, dt=dt_n, P=P, t=t, t_end=t_end)
        t += dt
        used.append(dt)
    return u, t, used


def rk3_amplification(z: complex) -> complex:
    """Stability polynomial of SSP-RK3 for u' = z u / dt: 1 + z + z^2/2 + z^3/6."""
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


# ---------------------------------------------------------------- sparse fields

def nonlinear_by_convolution(uhat: np.ndarray, prm: Params, chunk_pairs: int = 1 << 22) -> np.ndarray:
    """b_hat of the divergence form from the Galerkin definition of the
    truncated product, B_hat_k = sum_{p + q = k} u_hat_p (x) u_hat_q over the
    full spectrum, for k in K_N.  Cost grows with the square of the number of
    nonzero modes: meant for sparse spectra at any N (no transform, no grid).
    The pairs (p, q) are visited row by row in blocks of about
    ``chunk_pairs``; every sum still adds its terms in the same order."""
    N = uhat.shape[-2]
    h = N // 2
    kx, ky, kz = wavenumbers(N)
    shape = (N, N, N // 2 + 1)
    m = np.any(uhat != 0, axis=0) & retained_mask(N)
    K = np.stack([np.broadcast_to(kx, shape)[m], np.broadcast_to(ky, shape)[m],
                  np.broadcast_to(kz, shape)[m]], axis=1)
    V = uhat[:, m].T                                   # (nmodes, 3)
    pos = K[:, 2] > 0                                  # mirror kz > 0 to -k
    K = np.concatenate([K, -K[pos]])
    V = np.concatenate([V, np.conj(V[pos])])
    n = len(K)
    B = np.zeros((3, 3) + shape, dtype=np.complex128)
    rows = max(1, chunk_pairs // max(n, 1))
    for i0 in range(0, n, rows):
        ksum = K[i0:i0 + rows, None, :] + K[None, :, :]      # (rows, n, 3)
        keep = (np.abs(ksum[..., 0]) < h) & (np.abs(ksum[..., 1]) < h) & \
               (ksum[..., 2] >= 0) & (ksum[..., 2] < h)
        ii, jj = np.nonzero(keep)
        ks = ksum[ii, jj]
        ii = ii + i0
        ix, iy, iz = ks[:, 0] % N, ks[:, 1] % N, ks[:, 2]
        for j in range(3):
            for l in range(3):
                np.add.at(B[j, l], (ix, iy, iz), V[ii, j] * V[jj, l])
    kap = kappa(N, prm.L)
    b = np.stack([-1j * sum(kap[l] * B[j, l] for l in range(3)) for j in range(3)])
    return b * retained_mask(N)


def rhs_by_convolution(uhat: np.ndarray, prm: Params) -> np.ndarray:
    """R(u_hat) with the nonlinear term from ``nonlinear_by_convolution``."""
    N = uhat.shape[-2]
    b = nonlinear_by_convolution(uhat, prm)
    return (leray(b, prm.L) - dissipation(N, prm) * uhat) * retained_mask(N)


def rhs_sparse(K: np.ndarray, V: np.ndarray, N: int, prm: Params):
    """R(u_hat) for a field given by its nonzero modes (K integer wave vectors
    with k_z >= 0 as stored in the D1 layout, V their coefficients), at any N
    without a grid: the Galerkin sum of ``nonlinear_by_convolution`` over mode
    pairs, evaluated only at the modes it reaches in K_N, the Leray
    projection, and -lambda_k u_hat_k at the input modes.  Returns (Kout, R):
    every mode where R can be nonzero (k_z >= 0) and R there."""
    h = N // 2
    K = np.asarray(K, dtype=np.int64).reshape(-1, 3)
    V = np.asarray(V, dtype=np.complex128).reshape(-1, 3)
    pos = K[:, 2] > 0                                  # a stored k_z > 0 mode stands for -k too
    Kf = np.concatenate([K, -K[pos]])
    Vf = np.concatenate([V, np.conj(V[pos])])
    ksum = (Kf[:, None, :] + Kf[None, :, :]).reshape(-1, 3)
    ii, jj = np.divmod(np.arange(len(Kf) ** 2), len(Kf))
    keep = (np.abs(ksum[:, 0]) < h) & (np.abs(ksum[:, 1]) < h) & (ksum[:, 2] >= 0) & (ksum[:, 2] < h)
    ks, ii, jj = ksum[keep], ii[keep], jj[keep]
    inband = np.all(np.abs(K[:, :2]) < h, axis=1) & (K[:, 2] < h)
    Kout, inv = np.unique(np.concatenate([ks, K[inband]]), axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    Bsum = np.zeros((len(Kout), 3, 3), dtype=np.complex128)
    np.add.at(Bsum, inv[:len(ks)], Vf[ii][:, :, None] * Vf[jj][:, None, :])
    kap = (TWO_PI / prm.L) * Kout.astype(np.float64)
    b = -1j * np.einsum("nl,njl->nj", kap, Bsum)
    k2 = np.sum(kap * kap, axis=1)
    safe = np.where(k2 > 0, k2, 1.0)
    R = b - kap * (np.sum(kap * b, axis=1) / safe)[:, None]
    R[k2 == 0] = 0.0
    kin = Kout[inv[len(ks):]]
    lam = dissipation_of_k2(np.sum(kin * kin, axis=1), N, prm)
    np.add.at(R, inv[len(ks):], -lam[:, None] * V[inband])
    return Kout, R
