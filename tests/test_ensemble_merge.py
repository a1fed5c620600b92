"""Host logic of sharded ensembles: the Chan merge of shard statistics equals
the statistics of the whole ensemble, in one process and across two gloo
ranks (the multi-GPU path: members shard, statistics merge at output times)."""
import os

import numpy as np
import pytest

import ns3d_inputs as I
from oracle import stats as T
from paper_2401_09843_gb300.ensemble import allreduce_stats, merge_stats

L = 2 * np.pi


def _members(N=8, M=7):
    return np.stack([I.random_spectrum(N, seed=31, member=m, k0=2.0) for m in range(M)])


def _as_api(st):
    """oracle.stats dict -> the keys Plan.ensemble_stats returns."""
    return {"members": st["M"], "mean": st["mean"], "second": st["second"], "var": st["var"],
            "spectrum": st["spectrum"], "spectrum_se": st["spectrum_stderr"],
            "s2": st["s2"], "s2_se": st["s2_stderr"],
            "s2_ball": st["s2_ball"], "s2_ball_se": st["s2_ball_stderr"],
            "energy": st["energy"], "energy_se": st["energy_stderr"]}


def _close(a, b):
    for k in ("mean", "second", "var", "spectrum", "spectrum_se", "s2", "s2_se", "s2_ball", "s2_ball_se",
              "energy", "energy_se"):
        assert np.allclose(a[k], b[k], rtol=1e-11, atol=1e-14), k
    assert a["members"] == b["members"]


@pytest.mark.parametrize("split", [1, 3, 6])
def test_merge_equals_whole(split):
    u = _members()
    whole = _as_api(T.ensemble_stats(u, L))
    part = merge_stats(_as_api(T.ensemble_stats(u[:split], L)), _as_api(T.ensemble_stats(u[split:], L)))
    _close(part, whole)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u = _members()
    shard = u[rank::world]
    merged = allreduce_stats(_as_api(T.ensemble_stats(shard, L)))
    q.put((rank, merged))
    dist.destroy_process_group()


def test_two_rank_gloo_merge():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = _as_api(T.ensemble_stats(_members(), L))
    for r in (0, 1):
        _close(res[r], whole)
