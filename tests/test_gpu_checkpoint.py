"""Stop and resume through a checkpoint file: a run resumed in a new plan
continues bit for bit (state, time, step count), on the fused FP32 path,
the generic FP32 path and FP64, with CFL steps and a t_end clip."""
import numpy as np
import pytest

import ns3d_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B(lib):
    from paper_2401_09843_gb300 import binding
    return binding


@pytest.mark.parametrize("N,dt", [(64, "f32"), (24, "f32"), (32, "f64")])
def test_resume_is_bitwise(B, tmp_path, N, dt):
    from paper_2401_09843_gb300 import checkpoint as C
    dtype = B.NS3D_F32 if dt == "f32" else B.NS3D_F64
    kw = dict(eps0=1.0, cfl=0.5, nu=0.002)
    u0 = I.random_spectrum(N, seed=N + 11, k0=3.0)
    a = B.Plan([N, N], dtype, **kw)
    a.set_initial(0, u0)
    a.set_initial(1, 0.5 * u0)
    a.step(3, t_end=0.2)
    path = str(tmp_path / "ckp")
    head = C.save(a, 0, path, seed=N + 11)
    assert head["nsteps"] == 3 and head["t"] > 0
    a.step(4, t_end=0.2)
    ref, tref = a.get_state_host(0)
    nref = a.clock(0)[1]
    a.close()
    b = B.Plan([N], dtype, **kw)
    C.restore(b, 0, path)
    b.step(4, t_end=0.2)
    got, t = b.get_state_host(0)
    assert np.array_equal(got, ref) and t == tref and b.clock(0)[1] == nref
    b.close()
    with pytest.raises(ValueError):
        c = B.Plan([N], dtype, eps0=2.0)
        try:
            C.restore(c, 0, path)
        finally:
            c.close()
