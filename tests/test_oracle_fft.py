"""Pins for the oracle's own FFT: brute-force DFT, Parseval, inverse, deltas.

The brute-force sums here are written from the DFT definition
X[k] = sum_j x[j] exp(-2 pi i k.j / n) with the exponent formed from the full
multi-index (not as a product of 1D transforms), so they share nothing with
the recursive factorisation in oracle.fft."""
import itertools

import numpy as np
import pytest

from oracle import fft as F


def brute_1d(x, sign=-1):
    n = len(x)
    return np.array([sum(x[j] * np.exp(sign * 2j * np.pi * j * k / n) for j in range(n))
                     for k in range(n)])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 12, 13, 15, 16, 18, 24, 25,
                               35, 36, 48, 49, 96])
def test_fft_matches_brute_1d(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        ref = brute_1d(x, sign)
        got = F.fft(x, sign)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def brute_nd(x, sign=-1):
    shape = x.shape
    idx = np.array(list(itertools.product(*[range(s) for s in shape])))     # (M, d)
    phase = np.zeros((len(idx), len(idx)))
    for d, s in enumerate(shape):
        phase += np.outer(idx[:, d], idx[:, d]) / s
    W = np.exp(sign * 2j * np.pi * phase)
    return (W @ x.ravel()).reshape(shape)


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 8, 3), (12, 12, 12), (16, 16, 16), (9, 10, 14)])
def test_fftn_matches_brute_3d(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = brute_nd(x)
    got = F.fftn(x, axes=(0, 1, 2))
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_parseval_and_inverse():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 48)) + 1j * rng.standard_normal((5, 48))
    X = F.fft(x)
    assert np.allclose(np.sum(np.abs(X) ** 2, -1), 48 * np.sum(np.abs(x) ** 2, -1), rtol=1e-13)
    assert np.allclose(F.fft(X, +1) / 48, x, atol=1e-14)


def test_single_mode_is_delta():
    n = 24
    for m in (0, 1, 5, 12, 23):
        x = np.exp(2j * np.pi * m * np.arange(n) / n)
        X = F.fft(x)
        ref = np.zeros(n, complex)
        ref[m] = n
        assert np.max(np.abs(X - ref)) < 1e-12


@pytest.mark.parametrize("n", [6, 8, 12, 15, 48])
def test_real_transforms_by_definition(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n))
    Xh = F.rfft_last(x)
    assert Xh.shape == (3, n // 2 + 1)
    ref = np.stack([brute_1d(r)[: n // 2 + 1] for r in x])
    assert np.max(np.abs(Xh - ref)) < 1e-12
    assert np.allclose(F.irfft_last(Xh, n) / n, x, atol=1e-14)
