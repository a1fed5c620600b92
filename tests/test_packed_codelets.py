"""The packed in-register DFTs (codelets_packed.cuh) on the CPU, through the
kernel emulator: for every radix and both signs, two independent transforms in
lockstep (one per lane of a float pair) and the one-lane float version, each
against the DFT written out from its definition in FP64.  The lanes must not
mix: transforming a pair gives each lane's own transform bit for bit."""
import ctypes

import numpy as np
import pytest

RADICES = [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 32]


@pytest.fixture(scope="module")
def hc():
    from paper_2401_09843_gb300 import build
    lib = ctypes.CDLL(build.build_hostcheck())
    lib.ns3d_hostcheck_dftp.restype = ctypes.c_int
    lib.ns3d_hostcheck_dftp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p]
    return lib


def dft_definition(x, sign):
    n = len(x)
    j = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return W @ x            # X[k] = sum_j x[j] exp(sign 2 pi i j k / n)


def run(hc, R, sign, xs):
    """xs: list of 1 or 2 complex vectors (lanes)."""
    lanes = len(xs)
    re = np.ascontiguousarray(np.stack([x.real for x in xs], axis=-1).astype(np.float32))
    im = np.ascontiguousarray(np.stack([x.imag for x in xs], axis=-1).astype(np.float32))
    assert hc.ns3d_hostcheck_dftp(R, sign, lanes, re.ctypes.data, im.ctypes.data) == 0
    return [re[:, l].astype(np.float64) + 1j * im[:, l].astype(np.float64) for l in range(lanes)]


@pytest.mark.parametrize("R", RADICES)
@pytest.mark.parametrize("sign", [-1, 1])
def test_packed_codelet_matches_definition(hc, R, sign):
    rng = np.random.default_rng(1000 * R + (sign > 0))
    a = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    b = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    a32 = a.astype(np.complex64).astype(np.complex128)
    b32 = b.astype(np.complex64).astype(np.complex128)
    pa, pb = run(hc, R, sign, [a32, b32])
    for got, x in ((pa, a32), (pb, b32)):
        ref = dft_definition(x, sign)
        assert np.linalg.norm(got - ref) < 4e-7 * np.log2(2 * R) * np.linalg.norm(ref)
    # lanes are independent: the pair equals each lane run alone, bit for bit
    (sa,) = run(hc, R, sign, [a32])
    assert np.array_equal(sa, pa)
    (sb,) = run(hc, R, sign, [b32])
    assert np.array_equal(sb, pb)


def test_packed_codelet_unit_impulses(hc):
    """A unit impulse at j gives the pure exponential exp(sign 2 pi i j k / R)."""
    for R in (12, 16, 24, 32):
        for j in (0, 1, R - 1):
            x = np.zeros(R, complex)
            x[j] = 1.0
            (got,) = run(hc, R, -1, [x])
            ref = np.exp(-2j * np.pi * j * np.arange(R) / R)
            assert np.max(np.abs(got - ref)) < 2e-7
    assert hc.ns3d_hostcheck_dftp(11, -1, 1, np.zeros(11, np.float32).ctypes.data,
                                  np.zeros(11, np.float32).ctypes.data) == -1
