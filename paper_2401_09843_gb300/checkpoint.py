"""Checkpoint files for one ensemble member (the paper's full-field writer,
section 2.4, used to stop and resume a run).

File layout (little-endian):
    8 bytes   magic b"NS3DCKP1"
    4 bytes   uint32 length n of the header
    n bytes   UTF-8 JSON header: N, dtype ("f32" | "f64"), t, nsteps, the
              solver parameters, and free-form metadata (e.g. the seed)
    body      the coefficients in the D1 layout [3][N][N][N/2 + 1], complex64
              or complex128, C order

Restoring a member with ``restore`` sets its state and its clock, so the run
continues bit for bit as if it had not stopped (same plan parameters).
"""
from __future__ import annotations

import ctypes
import json
import struct

import numpy as np

MAGIC = b"NS3DCKP1"
_DTYPES = {"f32": np.complex64, "f64": np.complex128}


def write_file(path: str, header: dict, uhat: np.ndarray) -> None:
    """Write a checkpoint: header (JSON-serialisable, with N and dtype) and
    the D1-layout coefficients."""
    N = int(header["N"])
    dt = _DTYPES[header["dtype"]]
    body = np.ascontiguousarray(uhat, dtype=dt)
    if body.shape != (3, N, N, N // 2 + 1):
        raise ValueError(f"coefficients of shape {body.shape} for N = {N}")
    head = json.dumps(header, sort_keys=True).encode("utf-8")
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(head)))
        f.write(head)
        f.write(body.astype(body.dtype.newbyteorder("<"), copy=False).tobytes())


def read_file(path: str):
    """(header, coefficients) of a checkpoint file."""
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a checkpoint file")
        (n,) = struct.unpack("<I", f.read(4))
        header = json.loads(f.read(n).decode("utf-8"))
        N = int(header["N"])
        dt = np.dtype(_DTYPES[header["dtype"]]).newbyteorder("<")
        count = 3 * N * N * (N // 2 + 1)
        body = np.frombuffer(f.read(count * dt.itemsize), dtype=dt, count=count)
    return header, body.reshape(3, N, N, N // 2 + 1).astype(dt.newbyteorder("="))


def _params_dict(plan) -> dict:
    p = plan.params
    return {name: getattr(p, name) for name, _ in p._fields_}


def save(plan, member: int, path: str, **meta) -> dict:
    """Checkpoint member `member` of a Plan (synchronises); returns the header."""
    from .binding import NS3D_F32
    uhat, _ = plan.get_state_host(member)
    t, nsteps = plan.clock(member)
    header = {"N": plan.N[member], "dtype": "f32" if plan.dtype == NS3D_F32 else "f64",
              "t": t, "nsteps": nsteps, "params": _params_dict(plan), "meta": meta}
    write_file(path, header, uhat)
    return header


def restore(plan, member: int, path: str) -> dict:
    """Set member `member` of a Plan from a checkpoint (state and clock); the
    plan must have the member's N, the file's dtype and the same parameters."""
    from .binding import NS3D_F32
    header, uhat = read_file(path)
    dtype = "f32" if plan.dtype == NS3D_F32 else "f64"
    if header["N"] != plan.N[member] or header["dtype"] != dtype:
        raise ValueError(f"checkpoint is {header['N']}^3 {header['dtype']}, member is "
                         f"{plan.N[member]}^3 {dtype}")
    mine = _params_dict(plan)
    for k, v in header["params"].items():
        if k in mine and mine[k] != v:
            raise ValueError(f"parameter {k}: checkpoint {v}, plan {mine[k]}")
    plan.set_initial_host(member, uhat)
    plan.set_clock(member, header["t"], header["nsteps"])
    return header
