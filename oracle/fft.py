"""Own FFT for the oracle (test infrastructure only).

The paper assumes FFTW/cuFFT for its transforms (section 3.1); the oracle
uses none of them.  ``fft`` below is the textbook recursive Cooley-Tukey
decimation in time for a length n = p m with p the smallest prime factor:

    X[k] = sum_{r<p} w_n^{r k} Y_r[k mod m],   Y_r = DFT_m(x[r::p]),
    w_n = exp(sign 2 pi i / n),

with the direct O(n^2) sum for a prime n.  Real transforms follow their
definitions: ``rfft`` keeps k = 0..n/2 of the complex transform of real data,
``irfft`` extends a half spectrum by X[n-k] = conj(X[k]) and keeps the real
part.  No transform here is normalised; callers scale.
"""
from __future__ import annotations

import numpy as np

__all__ = ["fft", "fft_axis", "fftn", "rfft_last", "irfft_last", "dft_direct"]


def _smallest_prime_factor(n: int) -> int:
    for p in (2, 3, 5, 7):
        if n % p == 0:
            return p
    f = 11
    while f * f <= n:
        if n % f == 0:
            return f
        f += 2
    return n


def _twiddle(e: np.ndarray, n: int, sign: int) -> np.ndarray:
    """exp(sign 2 pi i e / n) with the exponent reduced mod n first."""
    ang = (2.0 * np.pi / n) * (np.asarray(e) % n)
    return np.cos(ang) + sign * 1j * np.sin(ang)


def dft_direct(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Direct DFT along the last axis (the brute-force definition)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    j = np.arange(n)
    W = _twiddle(np.outer(j, j), n, sign)
    return x @ W


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT along the last axis, X[k] = sum_j x[j] w_n^{jk}.

    Decimation in time with n = p m: the p sub-sequences x[r::p] are
    transformed together (one recursive call on an (..., p, m) array), then
    for k = k1 + m k2
        X[k1 + m k2] = sum_r w_p^{r k2} (w_n^{r k1} Y_r[k1]),
    i.e. a twiddle multiply followed by a p-point DFT across r."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    p = _smallest_prime_factor(n)
    if p == n:
        return dft_direct(x, sign)
    m = n // p
    sub = np.swapaxes(x.reshape(x.shape[:-1] + (m, p)), -1, -2)     # [..., r, j] = x[j p + r]
    Y = fft(sub, sign)                                               # [..., r, k1]
    r = np.arange(p)[:, None]
    k1 = np.arange(m)[None, :]
    T = Y * _twiddle(r * k1, n, sign)
    Wp = _twiddle(np.outer(np.arange(p), np.arange(p)), p, sign)     # [k2, r]
    X = np.matmul(Wp, T)                                             # [..., k2, k1]
    return X.reshape(x.shape[:-1] + (n,))


def fft_axis(x: np.ndarray, axis: int, sign: int = -1) -> np.ndarray:
    """``fft`` applied along ``axis``."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(fft(x, sign), -1, axis)


def fftn(x: np.ndarray, axes, sign: int = -1) -> np.ndarray:
    """Unnormalised multi-dimensional DFT over ``axes``, one axis at a time."""
    y = np.asarray(x, dtype=np.complex128)
    for a in axes:
        y = fft_axis(y, a, sign)
    return y


def rfft_last(x: np.ndarray) -> np.ndarray:
    """Forward transform of real data along the last axis, k = 0..n/2."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[-1]
    return fft(x.astype(np.complex128), -1)[..., : n // 2 + 1]


def irfft_last(X: np.ndarray, n: int) -> np.ndarray:
    """Inverse of a half spectrum (k = 0..n/2) to n real samples: the missing
    k = n/2+1..n-1 are conj(X[n-k]); the result is the real part of the
    unnormalised inverse DFT."""
    X = np.asarray(X, dtype=np.complex128)
    h = X.shape[-1]
    full = np.zeros(X.shape[:-1] + (n,), dtype=np.complex128)
    full[..., :h] = X
    for k in range(h, n):
        full[..., k] = np.conj(X[..., n - k])
    return fft(full, +1).real
