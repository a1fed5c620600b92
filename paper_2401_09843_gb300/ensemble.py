"""Monte Carlo ensembles split across GPUs or processes (Algorithm 1).

Samples are independent, so an ensemble shards with no data-path exchange:
each rank advances its own members and computes the statistics of its shard
with ``Plan.ensemble_stats``.  The only communication is the merge of those
statistics at output times, done here on the host with the pairwise formula of
Chan, Golub and LeVeque for (count, mean, sum of squared deviations):

    n = n_a + n_b,  mean = mean_a + (mean_b - mean_a) n_b / n,
    M2 = M2_a + M2_b + (mean_b - mean_a)^2 n_a n_b / n.

Standard errors are sqrt(M2 / (n - 1) / n); pointwise second moments are means
of products and merge as count-weighted means.
"""
from __future__ import annotations

import numpy as np

_PAIRS = ["spectrum", "s2", "s2_ball", "energy", "enstrophy_spectrum", "enstrophy", "dissipation"]


def _m2_from_se(se, n):
    """Sum of squared deviations from a standard error sqrt(M2/(n-1)/n)."""
    se = np.asarray(se, dtype=np.float64)
    return se * se * n * (n - 1) if n > 1 else np.zeros_like(se)


def _se_from_m2(m2, n):
    return np.sqrt(m2 / (n - 1) / n) if n > 1 else np.zeros_like(np.asarray(m2, dtype=np.float64))


def merge_stats(a: dict, b: dict) -> dict:
    """Merge the statistics of two disjoint member sets of one level."""
    na, nb = int(a["members"]), int(b["members"])
    if na == 0:
        return dict(b)
    if nb == 0:
        return dict(a)
    n = na + nb
    out = {"members": n}
    for key in _PAIRS:
        if key not in a or key not in b:
            continue
        se_key = key + "_se"
        ma, mb = np.asarray(a[key], dtype=np.float64), np.asarray(b[key], dtype=np.float64)
        d = mb - ma
        mean = ma + d * (nb / n)
        m2 = _m2_from_se(a[se_key], na) + _m2_from_se(b[se_key], nb) + d * d * (na * nb / n)
        out[key] = mean if mean.ndim else float(mean)
        se = _se_from_m2(m2, n)
        out[se_key] = se if np.ndim(se) else float(se)
    if "mean" in a and "mean" in b:
        ma, mb = a["mean"], b["mean"]
        d = mb - ma
        out["mean"] = ma + d * (nb / n)
        va = a["var"] * (na - 1) if na > 1 else np.zeros_like(a["var"])
        vb = b["var"] * (nb - 1) if nb > 1 else np.zeros_like(b["var"])
        out["var"] = (va + vb + d * d * (na * nb / n)) / (n - 1)
        out["second"] = (na * a["second"] + nb * b["second"]) / n
    return out


def allreduce_stats(stats: dict, group=None) -> dict:
    """Merge every rank's shard statistics (torch.distributed, any backend);
    every rank returns the statistics of the whole ensemble."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, stats, group=group)
    acc = parts[0]
    for p in parts[1:]:
        acc = merge_stats(acc, p)
    return acc


def wasserstein1_one_point(sa, sb) -> float:
    """1-point Wasserstein distance between two ensembles of fields on the same
    points (mesh-refinement studies, section 6.1): the mean over the points of
    W1 between the empirical one-point marginals.  sa (Ma, ...), sb (Mb, ...).
    Equal sample counts use the sorted-sample form mean |a_(i) - b_(i)|; other
    counts integrate |F_a - F_b| between the merged sorted samples."""
    a = np.sort(np.asarray(sa, dtype=np.float64).reshape(np.shape(sa)[0], -1), axis=0)
    b = np.sort(np.asarray(sb, dtype=np.float64).reshape(np.shape(sb)[0], -1), axis=0)
    if a.shape[0] == b.shape[0]:
        return float(np.mean(np.abs(a - b)))
    t = np.sort(np.concatenate([a, b], axis=0), axis=0)              # (Ma + Mb, points)
    lo, dt = t[:-1], np.diff(t, axis=0)
    Fa = np.stack([np.sum(a <= x[None, :], axis=0) for x in lo]) / a.shape[0]
    Fb = np.stack([np.sum(b <= x[None, :], axis=0) for x in lo]) / b.shape[0]
    return float(np.mean(np.sum(np.abs(Fa - Fb) * dt, axis=0)))
