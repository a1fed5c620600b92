"""GPU parity of the advective (nonlinear_form = 1) and rotational
(nonlinear_form = 2) forms of the nonlinear term, through the C ABI, against
the oracle's forms (relative L2 <= 1e-11 in FP64, <= 2e-5 in FP32, as for the
divergence form).  For a divergence-free field with 3/2 padding the three
forms agree after the Leray projection up to rounding, so at 256^3 the forms
are checked against the divergence form's own GPU path."""
import numpy as np
import pytest

import ns3d_inputs as I
from oracle import solver as S

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-11, 2e-5


def rel(a, b):
    a = np.asarray(a)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel())


@pytest.fixture(scope="module")
def B(lib):
    from paper_2401_09843_gb300 import binding
    return binding


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_form_rhs_matches_oracle(B, form, dt):
    """Several levels in one plan (ragged z tiles at N = 24 and 40, radix 5 at
    P = 60); each member's RHS against the oracle's RHS in the same form."""
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    Ns = [16, 24, 40, 64, 24]
    prm = S.Params(nu=0.01, eps0=1.0, L=5.0, nonlinear_form=form)
    p = B.Plan(Ns, dtype, nu=0.01, eps0=1.0, L=5.0, nonlinear_form=form)
    for m, N in enumerate(Ns):
        uh = I.random_spectrum(N, seed=300 + 10 * form + m, k0=2.5)
        got = p.eval_rhs(m, uh).cpu().numpy()
        P = p.info(m)["P"]
        assert P == S.padded_size(N)
        ref = S.rhs(uh, prm, P=P)
        assert rel(got, ref) < (TOL64 if dt == "f64" else TOL32), (m, N)
        h = N // 2
        assert np.all(got[:, h] == 0) and np.all(got[:, :, h] == 0) and np.all(got[..., h] == 0)
    p.close()


@pytest.mark.parametrize("form", [1, 2])
def test_form_rhs_fp64_at_96(B, form):
    N = 96
    prm = S.Params(eps0=1.0, nonlinear_form=form)
    uh = I.random_spectrum(N, seed=form, k0=8.0)
    p = B.Plan([N], B.NS3D_F64, eps0=1.0, nonlinear_form=form)
    got = p.eval_rhs(0, uh).cpu().numpy()
    assert rel(got, S.rhs(uh, prm, P=p.info(0)["P"])) < TOL64
    p.close()


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_form_cfl_steps_match_oracle(B, form, dt):
    """CFL steps in the form: the CFL maximum comes from the form's z pass."""
    N = 32
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    prm = S.Params(cfl=0.5, eps0=1.0, nonlinear_form=form)
    u0 = I.random_spectrum(N, seed=20240001)
    p = B.Plan([N], dtype, cfl=0.5, eps0=1.0, nonlinear_form=form)
    p.set_initial(0, u0)
    p.step(5)
    got, t = p.get_state(0, with_time=True)
    ref, tref, _ = S.integrate(u0, prm, 5, P=p.info(0)["P"])
    assert abs(t - tref) < (1e-13 if dt == "f64" else 1e-6) * tref
    assert rel(got.cpu().numpy(), ref) < (TOL64 if dt == "f64" else TOL32)
    p.close()


def test_forms_agree_with_divergence_form_at_256(B):
    """Full size, FP32: the three forms' GPU paths give the same RHS up to
    FP32 rounding, and the same five CFL steps."""
    N = 256
    u0 = I.random_spectrum(N, seed=20240001)
    out = {}
    for form in (0, 1, 2):
        p = B.Plan([N], B.NS3D_F32, cfl=0.5, eps0=1.0, nonlinear_form=form)
        assert p.info(0)["P"] == 384
        r = p.eval_rhs(0, u0).cpu().numpy()
        p.set_initial(0, u0)
        p.step(5)
        s, t = p.get_state(0, with_time=True)
        out[form] = (r, s.cpu().numpy(), t)
        p.close()
    for form in (1, 2):
        assert rel(out[form][0], out[0][0]) < TOL32, form
        assert rel(out[form][1], out[0][1]) < TOL32, form
        assert abs(out[form][2] - out[0][2]) < 1e-6 * out[0][2]


@pytest.mark.parametrize("form", [1, 2])
def test_form_nonfinite_sets_status(B, form):
    N = 16
    u = I.random_spectrum(N, seed=1, k0=2.0)
    u[0, 1, 2, 3] = np.nan
    p = B.Plan([N], B.NS3D_F64, eps0=1.0, nonlinear_form=form)
    p.set_initial(0, u)
    p.step(1)
    with pytest.raises(B.Ns3dError) as e:
        p.synchronize()
    assert e.value.code == 4
    p.close()


@pytest.mark.parametrize("form", [1, 2])
def test_form_plan_gradient(B, form):
    """The band-energy gradient of a form-1/2 plan (forward stages recomputed
    in that form, the transpose of the divergence form's linearisation) equals
    the divergence form's gradient and the oracle's, up to rounding."""
    from oracle import adjoint as A
    N, dt, n = 12, 0.04, 6
    prm = S.Params(nu=0.01, eps0=1.0)
    u0 = I.random_spectrum(N, seed=8, k0=2.5)
    p = B.Plan([N], B.NS3D_F64, nu=0.01, eps0=1.0, dt_fixed=dt, nonlinear_form=form)
    p.set_initial(0, u0)
    got = p.grad_band_energy(0, 2.0, 4.0, n, checkpoint_every=4).cpu().numpy()
    p.close()
    ref = A.grad_band_energy(u0, prm, n, dt, 2.0, 4.0, checkpoint_every=4)
    assert rel(got, ref) < 1e-11


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_form_rhs_full_size_sparse_spectrum(B, form, dt):
    """256^3 in the production launch shapes (FP32 rotational form: the
    register-resident z pass; otherwise the tuned tile kernel) against the
    truncated product of a divergence-free sparse field summed over mode
    pairs, which every form equals after the projection."""
    N = 256
    dtype = B.NS3D_F64 if dt == "f64" else B.NS3D_F32
    prm = S.Params(nu=0.0, eps0=1.0)
    uh = I.sparse_random(N, seed=N + 7 + form, nmodes=48)
    ref = S.rhs_by_convolution(uh, prm)
    p = B.Plan([N], dtype, nu=0.0, eps0=1.0, nonlinear_form=form)
    got = p.eval_rhs(0, uh).cpu().numpy()
    p.close()
    assert rel(got, ref) < (TOL64 if dt == "f64" else TOL32)


def test_rotational_register_kernel_two_members(B):
    """Two members in one level at a register size (FP32, P = 48): each
    member's RHS and CFL steps (per-member dt from the kernel's CFL maximum)
    against the oracle."""
    N = 32
    prm = S.Params(cfl=0.5, eps0=1.0, nonlinear_form=2)
    u0 = [I.random_spectrum(N, seed=70 + m, k0=2.0 + m) for m in range(2)]
    p = B.Plan([N, N], B.NS3D_F32, cfl=0.5, eps0=1.0, nonlinear_form=2)
    for m in range(2):
        assert rel(p.eval_rhs(m, u0[m]).cpu().numpy(), S.rhs(u0[m], prm, P=48)) < TOL32, m
        p.set_initial(m, u0[m])
    p.step(3)
    for m in range(2):
        got, t = p.get_state(m, with_time=True)
        ref, tref, _ = S.integrate(u0[m], prm, 3, P=48)
        assert abs(t - tref) < 1e-6 * tref, m
        assert rel(got.cpu().numpy(), ref) < TOL32, m
    p.close()
