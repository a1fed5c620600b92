"""Checkpoint file format (host only): round trip, header checks."""
import numpy as np
import pytest

import ns3d_inputs as I
from paper_2401_09843_gb300 import checkpoint as C


@pytest.mark.parametrize("dtype,npd", [("f32", np.complex64), ("f64", np.complex128)])
def test_round_trip_is_exact(tmp_path, dtype, npd):
    N = 12
    u = I.random_spectrum(N, seed=4).astype(npd)
    head = {"N": N, "dtype": dtype, "t": 0.125, "nsteps": 7, "params": {"nu": 0.01}, "meta": {"seed": 4}}
    path = str(tmp_path / "m0.ckp")
    C.write_file(path, head, u)
    h2, u2 = C.read_file(path)
    assert h2 == head
    assert u2.dtype == npd and np.array_equal(u2, u)


def test_rejects_wrong_shape_and_magic(tmp_path):
    with pytest.raises(ValueError):
        C.write_file(str(tmp_path / "x"), {"N": 8, "dtype": "f64"}, np.zeros((3, 8, 8, 4), complex))
    bad = tmp_path / "bad"
    bad.write_bytes(b"NOTACKPT" + b"\0" * 16)
    with pytest.raises(ValueError):
        C.read_file(str(bad))
