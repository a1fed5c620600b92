"""The allocation-free right-hand side (ns3d_eval_rhs_noalloc) against the
plan-based one (ns3d_eval_rhs) and the oracle, through the C ABI, on two calls
in a row.

It serves callers that may not allocate device memory when they need the
derivative (a device memory budget fixed at start-up, a plug-in that must not
re-enter its host's allocator, a loop that cannot afford cudaMalloc's device
synchronisation): all its intermediates live in the library's fixed device
array, so two calls in a row also check that the second call is not disturbed
by what the first left there.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_rhs_matches_plan_rhs_twice(lib, N, dt):
    import torch
    from paper_2401_09843_gb300 import binding as B
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    tol = 1e-11 if dt == "f64" else 2e-5
    prm = B.default_params(nu=0.01, eps0=1.0)
    plan = B.Plan([N], dtype, params=prm)
    oprm = S.Params(nu=0.01, eps0=1.0)
    for call, seed in enumerate((11, 12)):
        uh = I.random_spectrum(N, seed=seed, k0=3.0)
        x = torch.from_numpy(uh).to(device="cuda", dtype=plan.cdtype)
        got = B.eval_rhs_noalloc(x, dtype, prm)
        ref = plan.eval_rhs(0, uh)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        assert rel(got, ref.cpu().numpy()) < tol, call
        assert rel(got.astype(np.complex128), S.rhs(uh, oprm)) < tol, call
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    import torch
    from paper_2401_09843_gb300 import binding as B
    lib_ = B.load()
    prm = B.default_params()
    x = torch.zeros((3, 64, 64, 33), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib_.ns3d_eval_rhs_noalloc(64, B.NS3D_F64, ctypes.byref(prm), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), s)
    assert rc == 1
    big = B.default_params(n_pad=64)
    x = torch.zeros((3, 32, 32, 17), dtype=torch.complex128, device="cuda")
    rc = lib_.ns3d_eval_rhs_noalloc(32, B.NS3D_F64, ctypes.byref(big), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), s)
    assert rc == 1


def test_noalloc_padding_choices(lib):
    """n_pad = -1 takes the smallest 7-smooth size like n_pad = 0 (for N = 22:
    P = 35, not 33 = 3 x 11); a given padded size with a prime factor above 7
    is NOT_SUPPORTED, like at plan creation."""
    import torch
    from paper_2401_09843_gb300 import binding as B
    lib_ = B.load()
    N = 22
    uh = I.random_spectrum(N, seed=21, k0=3.0)
    x = torch.from_numpy(uh).to(device="cuda", dtype=torch.complex128)
    a = B.eval_rhs_noalloc(x, B.NS3D_F64, B.default_params(eps0=1.0, n_pad=-1))
    b = B.eval_rhs_noalloc(x, B.NS3D_F64, B.default_params(eps0=1.0, n_pad=0))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert rel(a.cpu().numpy(), S.rhs(uh, S.Params(eps0=1.0))) < 1e-11
    y = torch.empty_like(x)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bad = B.default_params(n_pad=44)         # 44 = 4 x 11 >= 3N/2
    rc = lib_.ns3d_eval_rhs_noalloc(N, B.NS3D_F64, ctypes.byref(bad), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), s)
    assert rc == 7
    worse = B.default_params(n_pad=-2)
    rc = lib_.ns3d_eval_rhs_noalloc(N, B.NS3D_F64, ctypes.byref(worse), ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(y.data_ptr()), s)
    assert rc == 1
