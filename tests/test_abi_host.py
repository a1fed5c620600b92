"""Host-side checks of the library boundary (no GPU needed):
* libns3d.so builds, loads and exports every function include/ns3d.h declares;
* argument validation and the no-device error path return status codes;
* the CPU emulation of the kernels' block bodies (same source as the CUDA
  kernels, one emulated thread per block) matches the oracle: this pins the
  index logic -- strides, tiles, ragged tails, padding and truncation maps, the
  two-for-one real transforms, radix plans -- before any GPU run."""
import ctypes
import os
import re

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2401_09843_gb300 import build
    build.build_all()
    return build


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ns3d.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ns3d_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_header_function(built):
    from paper_2401_09843_gb300 import binding
    lib = binding.load()
    names = header_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.SYMBOLS) == names


def test_library_resolves_every_symbol_at_load(built):
    """Immediate binding: an undefined symbol (e.g. a kernel template that no
    translation unit instantiates) fails here, not on the GPU machine."""
    import os
    ctypes.CDLL(built.LIB, mode=os.RTLD_NOW | os.RTLD_LOCAL)


def test_status_strings_and_defaults(built):
    from paper_2401_09843_gb300 import binding
    lib = binding.load()
    assert lib.ns3d_status_string(0) == b"ok"
    assert lib.ns3d_status_string(7) == b"not supported"
    p = binding.default_params()
    assert abs(p.L - 2 * np.pi) < 1e-15 and p.s == 1.5 and p.theta == 0.5 and p.cfl == 0.5


def test_invalid_arguments_are_rejected(built):
    from paper_2401_09843_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    p = binding.default_params()
    ok = (ctypes.c_int * 1)(32)
    for bad in ([7], [0], [2], [-8]):
        arr = (ctypes.c_int * 1)(*bad)
        assert lib.ns3d_plan_create(ctypes.byref(h), arr, 1, 0, ctypes.byref(p), None, 0) == 1
    assert lib.ns3d_plan_create(ctypes.byref(h), ok, 0, 0, ctypes.byref(p), None, 0) == 1
    assert lib.ns3d_plan_create(ctypes.byref(h), ok, 1, 5, ctypes.byref(p), None, 0) == 1
    for form in (-1, 3):                               # 0, 1 and 2 are the three forms
        q = binding.default_params(nonlinear_form=form)
        assert lib.ns3d_plan_create(ctypes.byref(h), ok, 1, 0, ctypes.byref(q), None, 0) == 1
    q = binding.default_params(n_pad=40)              # below 3N/2 = 48: would alias
    assert lib.ns3d_plan_create(ctypes.byref(h), ok, 1, 0, ctypes.byref(q), None, 0) == 1
    q = binding.default_params(cfl=0.0)
    assert lib.ns3d_plan_create(ctypes.byref(h), ok, 1, 0, ctypes.byref(q), None, 0) == 1
    assert lib.ns3d_step(None, 1, 0.0) == 1
    assert lib.ns3d_set_initial(None, 0, None, 0) == 1


def test_no_device_returns_cuda_error(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2401_09843_gb300 import binding
    lib = binding.load()
    h = ctypes.c_void_p()
    p = binding.default_params()
    arr = (ctypes.c_int * 1)(32)
    assert lib.ns3d_plan_create(ctypes.byref(h), arr, 1, 0, ctypes.byref(p), None, 0) == 3


# --------------------------------------------------------------------------- CPU emulation

def hostcheck(built, uh, P, prm, nsteps=0, dt=0.0, dtype=1):
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_run.restype = ctypes.c_int
    cd = np.complex128 if dtype == 1 else np.complex64
    uin = np.ascontiguousarray(uh.astype(cd))
    uout = np.zeros_like(uin)
    p = np.array([prm.L, prm.nu, prm.s, prm.theta, prm.eps0, prm.mN_coef, prm.q_form, prm.cfl])
    t = ctypes.c_double(0)
    rc = lib.ns3d_hostcheck_run(dtype, uh.shape[-2], P, p.ctypes.data_as(ctypes.c_void_p),
                                uin.ctypes.data_as(ctypes.c_void_p), uout.ctypes.data_as(ctypes.c_void_p),
                                nsteps, ctypes.c_double(dt), ctypes.byref(t))
    return uout, rc, t.value


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("N,P", [(8, 12), (10, 15), (12, 18), (16, 24), (16, 32), (20, 30),
                                 (24, 36), (22, 35), (28, 42), (32, 48), (40, 60)])
def test_emulated_kernels_rhs_matches_oracle(built, N, P):
    prm = S.Params(nu=0.01, eps0=1.0, L=5.0)
    uh = I.random_spectrum(N, seed=N, k0=2.5)
    ref = S.rhs(uh, prm, P=P)
    got, rc, _ = hostcheck(built, uh, P, prm)
    assert rc == 0
    assert rel(got, ref) < 1e-13
    got32, _, _ = hostcheck(built, uh, P, prm, dtype=0)
    assert rel(got32, ref) < 2e-6


def test_emulated_kernels_steps_match_oracle(built):
    N, P = 16, 24
    prm = S.Params(nu=0.01, eps0=1.0, q_form=1)
    uh = I.random_spectrum(N, seed=3, k0=2.5)
    ref, _, _ = S.integrate(uh, prm.with_(dt_fixed=0.01), 3, P=P)
    got, rc, t = hostcheck(built, uh, P, prm, nsteps=3, dt=0.01)
    assert rc == 0 and abs(t - 0.03) < 1e-15
    assert rel(got, ref) < 1e-13
    # CFL step: the emulated kernels and the oracle take the same dt sequence
    ref, tref, _ = S.integrate(uh, prm, 2, P=P)
    got, rc, t = hostcheck(built, uh, P, prm, nsteps=2, dt=0.0)
    assert abs(t - tref) < 1e-14 and rel(got, ref) < 1e-12


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("N,P", [(8, 12), (10, 15), (16, 24), (22, 35), (32, 48), (24, 40)])
def test_emulated_nonlinear_forms_match_oracle(built, form, N, P):
    """The advective (1) and rotational (2) form paths of the kernels: the
    form's fields, their inverse passes, the z pass forming the products in
    shared memory, the forward passes and the spectral step, against the
    oracle's form and against the divergence form (equal after projection)."""
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_set_form(form)
    try:
        prm = S.Params(nu=0.01, eps0=1.0, L=5.0, nonlinear_form=form)
        uh = I.random_spectrum(N, seed=N + 7 * form, k0=2.5)
        ref = S.rhs(uh, prm, P=P)
        got, rc, _ = hostcheck(built, uh, P, prm)
        assert rc == 0
        assert rel(got, ref) < 1e-13
        assert rel(got, S.rhs(uh, prm, P=P, form=0)) < 1e-13
        got32, _, _ = hostcheck(built, uh, P, prm, dtype=0)
        assert rel(got32, ref) < 2e-6
        if N == 16:   # CFL steps: the same dt sequence as the oracle's
            ref, tref, _ = S.integrate(uh, prm, 2, P=P)
            got, rc, t = hostcheck(built, uh, P, prm, nsteps=2, dt=0.0)
            assert rc == 0 and abs(t - tref) < 1e-14 and rel(got, ref) < 1e-12
    finally:
        lib.ns3d_hostcheck_set_form(0)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("W", [1, 2, 8, 16])
def test_emulated_form_tile_shapes(built, form, W):
    """Every z tile width the plan's tuner may pick (ragged last tile at
    P = 24 with W = 16, odd P = 35) gives the oracle's RHS."""
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_set_form(form)
    lib.ns3d_hostcheck_set_form_tile(W)
    try:
        prm = S.Params(nu=0.01, eps0=1.0, nonlinear_form=form)
        for N, P in ((16, 24), (22, 35)):
            uh = I.random_spectrum(N, seed=5 * W + form, k0=2.5)
            got, rc, _ = hostcheck(built, uh, P, prm)
            assert rc == 0 and rel(got, S.rhs(uh, prm, P=P)) < 1e-13, (N, P)
    finally:
        lib.ns3d_hostcheck_set_form_tile(0)
        lib.ns3d_hostcheck_set_form(0)


def test_radix_plans(built):
    lib = ctypes.CDLL(built.HOSTLIB)
    r = (ctypes.c_int * 8)()
    for n in (12, 15, 48, 96, 192, 384, 768, 1152, 1536, 35, 49, 1000):
        k = lib.ns3d_hostcheck_plan(n, r, 8)
        assert k > 0 and int(np.prod([r[i] for i in range(k)])) == n
    assert lib.ns3d_hostcheck_plan(22, r, 8) == -1           # prime factor 11


@pytest.mark.parametrize("N,P", [(32, 48), (64, 96), (128, 192), (256, 384)])
def test_emulated_register_kernels_match_oracle(built, N, P):
    """The register-resident FP32 column and z passes (P = 48, 96, 192, 384 at
    the default padding P = 3N/2), emulated thread by thread, against the
    Galerkin product of a sparse field; then the generic kernels on the same
    input."""
    prm = S.Params(nu=0.01, eps0=1.0)
    uh = I.sparse_random(N, seed=P, nmodes=24)
    ref = S.rhs_by_convolution(uh, prm)          # the Galerkin product: independent of P
    got32, rc, _ = hostcheck(built, uh, P, prm, dtype=0)
    assert rc == 0 and rel(got32, ref) < 2e-6
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_use_fast(0)
    try:
        gen32, _, _ = hostcheck(built, uh, P, prm, dtype=0)
    finally:
        lib.ns3d_hostcheck_use_fast(1)
    assert rel(gen32, ref) < 2e-6


@pytest.mark.parametrize("N,P", [(32, 48), (64, 96), (128, 192), (256, 384)])
def test_emulated_rotational_register_z_pass(built, N, P):
    """The rotational form's register-resident z pass (FP32, P = 3N/2),
    emulated thread by thread, against the Galerkin product of a sparse field
    (equal for every form after the projection); then the tile kernel."""
    prm = S.Params(nu=0.01, eps0=1.0, nonlinear_form=2)
    uh = I.sparse_random(N, seed=P + 1, nmodes=24)
    ref = S.rhs_by_convolution(uh, prm)
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_set_form(2)
    try:
        got32, rc, _ = hostcheck(built, uh, P, prm, dtype=0)
        assert rc == 0 and rel(got32, ref) < 2e-6
        if N <= 64:
            lib.ns3d_hostcheck_use_fast(0)
            try:
                gen32, _, _ = hostcheck(built, uh, P, prm, dtype=0)
            finally:
                lib.ns3d_hostcheck_use_fast(1)
            assert rel(gen32, ref) < 2e-6
    finally:
        lib.ns3d_hostcheck_set_form(0)


@pytest.mark.parametrize("N", [32, 64])
def test_emulated_fused_x_steps_match_oracle(built, N):
    """Steps with the fused x pass (forward x + spectral + RK3 + next inverse x
    in one kernel; FP32, P = 3N/2), emulated thread by thread, against the
    oracle and against the unfused emulated kernels; CFL steps."""
    prm = S.Params(nu=0.005, eps0=1.0)
    uh = I.random_spectrum(N, seed=N + 1, k0=3.0)
    ref, tref, _ = S.integrate(uh, prm, 2)
    got, rc, t = hostcheck(built, uh, 3 * N // 2, prm, nsteps=2, dtype=0)
    assert rc == 0 and abs(t - tref) < 1e-6 * tref
    assert rel(got, ref) < 2e-5
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_use_fast(0)
    try:
        gen, _, tg = hostcheck(built, uh, 3 * N // 2, prm, nsteps=2, dtype=0)
    finally:
        lib.ns3d_hostcheck_use_fast(1)
    assert rel(got, gen) < 2e-6


@pytest.mark.parametrize("N", [128, 256])
def test_emulated_fused_x_large_tiles(built, N):
    """The fused x pass at P = 192 and 384 (radix 12 x 16 and 24 x 16),
    emulated thread by thread: one fixed-dt step of a sparse field against the
    unfused emulated kernels."""
    prm = S.Params(nu=0.01, eps0=1.0)
    uh = I.sparse_random(N, seed=N + 7, nmodes=24)
    got, rc, _ = hostcheck(built, uh, 3 * N // 2, prm, nsteps=1, dt=1e-3, dtype=0)
    assert rc == 0
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_use_fast(0)
    try:
        gen, _, _ = hostcheck(built, uh, 3 * N // 2, prm, nsteps=1, dt=1e-3, dtype=0)
    finally:
        lib.ns3d_hostcheck_use_fast(1)
    assert rel(got, gen) < 2e-6
    assert rel(got, uh) > 1e-6     # the step changed the field


@pytest.mark.parametrize("N,val", [(32, np.nan), (64, np.inf), (64, np.nan)])
def test_emulated_register_z_pass_flags_nonfinite(built, N, val):
    """A non-finite coefficient reaches every physical point of its line; the
    register-resident z pass (FP32) flags the member NONFINITE (bit 1)."""
    prm = S.Params(eps0=1.0)
    u = I.random_spectrum(N, seed=3, k0=3.0)
    u[1, 2, 3, 4] = val
    _, rc, _ = hostcheck(built, u, 3 * N // 2, prm, nsteps=1, dtype=0)
    assert rc & 1
    _, rc, _ = hostcheck(built, I.random_spectrum(N, seed=3, k0=3.0), 3 * N // 2, prm, nsteps=1,
                         dtype=0)
    assert rc == 0


@pytest.mark.parametrize("N", [32, 64, 128])
def test_emulated_three_pass_kernels_match_oracle(built, N):
    """The three-pass column and z kernels (the GPU builds them for P = 1536),
    emulated at short lengths P = 48 = 4x3x4, 96 = 6x4x4, 192 = 8x4x6 thread by
    thread: the RHS of a sparse field against the Galerkin product, and CFL
    steps against the oracle."""
    prm = S.Params(nu=0.01, eps0=1.0)
    uh = I.sparse_random(N, seed=N + 3, nmodes=24)
    ref = S.rhs_by_convolution(uh, prm)
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_use_fast(2)
    try:
        got, rc, _ = hostcheck(built, uh, 3 * N // 2, prm, dtype=0)
        assert rc == 0 and rel(got, ref) < 2e-6
        if N <= 64:
            u0 = I.random_spectrum(N, seed=N, k0=3.0)
            sref, tref, _ = S.integrate(u0, prm, 2)
            got, rc, t = hostcheck(built, u0, 3 * N // 2, prm, nsteps=2, dtype=0)
            assert rc == 0 and abs(t - tref) < 1e-6 * tref
            assert rel(got, sref) < 2e-5
    finally:
        lib.ns3d_hostcheck_use_fast(1)


@pytest.mark.parametrize("N", [32, 64])
def test_emulated_three_pass_kernels_fp64_double_single(built, N):
    """FP64 plans run their three-pass column and z kernels in double-single
    arithmetic (two FP32 per value, 48-bit significand): emulated at P = 48 =
    4x3x4 and 96 = 6x4x4 thread by thread, the RHS of a sparse field against
    the Galerkin product and two fixed steps against the oracle, both within
    the FP64 tolerance 1e-11 (the arithmetic's unit roundoff is 2^-48)."""
    prm = S.Params(nu=0.01, eps0=1.0)
    uh = I.sparse_random(N, seed=N + 11, nmodes=24)
    ref = S.rhs_by_convolution(uh, prm)
    lib = ctypes.CDLL(built.HOSTLIB)
    lib.ns3d_hostcheck_use_fast(2)
    try:
        got, rc, _ = hostcheck(built, uh, 3 * N // 2, prm, dtype=1)
        assert rc == 0 and rel(got, ref) < 1e-12, rel(got, ref)
        u0 = I.random_spectrum(N, seed=N + 1, k0=3.0)
        sref, _, _ = S.integrate(u0, prm.with_(dt_fixed=0.01), 2)
        got, rc, t = hostcheck(built, u0, 3 * N // 2, prm, nsteps=2, dt=0.01, dtype=1)
        assert rc == 0 and abs(t - 0.02) < 1e-15
        assert rel(got, sref) < 1e-12, rel(got, sref)
    finally:
        lib.ns3d_hostcheck_use_fast(1)


@pytest.mark.parametrize("sign", [1, -1])
def test_three_pass_column_block_1536(built, sign):
    """One column pass of the P = 1536 = 16x12x8 kernel (N = 1024), emulated:
    the padded inverse and the truncated forward against numpy's FFT, over a
    full 16-column tile and a ragged one."""
    P, N, h, ncols = 1536, 1024, 512, 21
    rng = np.random.default_rng(5)
    nin = N if sign > 0 else P
    x = (rng.standard_normal((nin, ncols)) + 1j * rng.standard_normal((nin, ncols))).astype(np.complex64)
    out = np.zeros((P if sign > 0 else N, ncols), np.complex64)
    lib = ctypes.CDLL(built.HOSTLIB)
    assert lib.ns3d_hostcheck_colpass3(sign, x.ctypes.data_as(ctypes.c_void_p),
                                       out.ctypes.data_as(ctypes.c_void_p), ncols) == 0
    xd = x.astype(np.complex128)
    if sign > 0:
        full = np.zeros((P, ncols), complex)
        full[:h] = xd[:h]
        full[P - N + h + 1:] = xd[h + 1:]       # rows h+1 .. N-1 are k = row - N
        ref = np.fft.ifft(full, axis=0) * P
    else:
        X = np.fft.fft(xd, axis=0)
        ref = np.zeros((N, ncols), complex)
        ref[:h] = X[:h]
        ref[h + 1:] = X[P - N + h + 1:]
    assert rel(out, ref) < 5e-6


def test_three_pass_z_block_1536(built):
    """The P = 1536 fused z pass on two x rows of a random Bq-like array,
    emulated: c2r of the three components, the six products, r2c truncated to
    kz < 512, against numpy's real FFTs; the CFL maximum too."""
    P, h, nx = 1536, 512, 2
    rng = np.random.default_rng(6)
    shape = (3, nx, P, h)
    bq = ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(P)).astype(np.complex64)
    out = np.zeros((6, nx, P, h), np.complex64)
    umax = ctypes.c_double()
    lib = ctypes.CDLL(built.HOSTLIB)
    rc = lib.ns3d_hostcheck_zpass3(bq.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                   nx, ctypes.byref(umax))
    assert rc == 0
    spec = np.zeros((3, nx, P, P // 2 + 1), complex)
    spec[..., :h] = bq
    u = np.fft.irfft(spec, n=P, axis=-1) * P          # ignores Im of kz = 0
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ref = np.stack([np.fft.rfft(u[j] * u[l], axis=-1)[..., :h] for j, l in pairs])
    assert rel(out, ref) < 5e-6
    umax_ref = np.max(np.abs(u[0]) + np.abs(u[1]) + np.abs(u[2]))
    assert abs(umax.value - umax_ref) < 1e-5 * umax_ref


@pytest.mark.parametrize("P,nx", [(384, 2), (1152, 1)])
def test_three_pass_z_block_fp64(built, P, nx):
    """The FP64 three-pass z pass (double-single arithmetic) at the padded sizes
    of the 256^3 and 768^3 FP64 workloads on a few x rows of random input,
    emulated: against numpy's FP64 real FFTs at the FP64 tolerance, and the
    CFL maximum."""
    h = P // 3
    rng = np.random.default_rng(P + 7)
    shape = (3, nx, P, h)
    bq = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(P)
    out = np.zeros((6, nx, P, h), np.complex128)
    umax = ctypes.c_double()
    lib = ctypes.CDLL(built.HOSTLIB)
    rc = lib.ns3d_hostcheck_zpass3_f64(P, bq.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                       nx, ctypes.byref(umax))
    assert rc == 0
    spec = np.zeros((3, nx, P, P // 2 + 1), complex)
    spec[..., :h] = bq
    u = np.fft.irfft(spec, n=P, axis=-1) * P          # ignores Im of kz = 0
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    ref = np.stack([np.fft.rfft(u[j] * u[l], axis=-1)[..., :h] for j, l in pairs])
    assert rel(out, ref) < 1e-12, rel(out, ref)
    umax_ref = np.max(np.abs(u[0]) + np.abs(u[1]) + np.abs(u[2]))
    assert abs(umax.value - umax_ref) < 1e-6 * umax_ref


@pytest.mark.parametrize("P", [48, 96])
def test_emulated_register_adjoint_z_pass_matches_tile_block(built, P):
    """The adjoint right-hand side's register-resident z pass (FP32; products
    c_j = sum_l u_l S_jl of the nine fields) against the generic tile block on
    the same random input, two x rows, emulated thread by thread; a field
    that is zero except one line changes only that line's outputs."""
    h, nx = P // 3, 2
    rng = np.random.default_rng(P)
    shape = (9, P, P, h)
    x = ((rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(P)).astype(np.complex64)
    fast = np.zeros((3, P, P, h), np.complex64)
    gen = np.zeros_like(fast)
    lib = ctypes.CDLL(built.HOSTLIB)
    rc = lib.ns3d_hostcheck_zadj(P, x.ctypes.data_as(ctypes.c_void_p), fast.ctypes.data_as(ctypes.c_void_p),
                                 gen.ctypes.data_as(ctypes.c_void_p), nx)
    assert rc == 0
    assert rel(fast[:, :nx], gen[:, :nx]) < 2e-6
    assert np.all(fast[:, nx:] == 0)
    # independent check of one column against numpy's real FFTs
    u = np.fft.irfft(np.concatenate([x[:, 1, 5].astype(complex), np.zeros((9, P // 2 + 1 - h))], axis=-1),
                     n=P, axis=-1) * P
    S = {(0, 0): u[3], (0, 1): u[4], (0, 2): u[5], (1, 1): u[6], (1, 2): u[7], (2, 2): u[8]}
    sym = lambda j, l: S[(min(j, l), max(j, l))]
    c = [sum(u[l] * sym(j, l) for l in range(3)) for j in range(3)]
    ref = np.stack([np.fft.rfft(cj)[:h] for cj in c])
    assert rel(fast[:, 1, 5], ref) < 2e-6
