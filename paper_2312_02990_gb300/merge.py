"""Merge of per-rank TTCF ensemble statistics (multi-GPU, weak scaling).

Each rank reduces its own mother groups on its GPU (``ttcf_response``); the
groups are independent, so the ensemble over all ranks follows from each
rank's per-sample group count n, mean and standard error.  Ranks exchange
those (a few arrays of S doubles) and fold them in rank order with the
pairwise update of Chan, Golub and LeVeque (1979):

    n = n_a + n_b,  d = m_b - m_a,  m = m_a + d n_b / n,
    M2 = M2_a + M2_b + d^2 n_a n_b / n,      with M2 = se^2 n (n - 1),

so the merged mean and standard error equal those of one run over all
groups (up to rounding), independently of the backend.
"""
from __future__ import annotations

import numpy as np

KEYS = ("corr", "dav", "ttcf")


def to_moments(resp: dict, n_groups: int) -> np.ndarray:
    """[len(KEYS), 3, S] array of (n, mean, M2) from a response dict."""
    S = len(resp["t"])
    out = np.zeros((len(KEYS), 3, S))
    for k, key in enumerate(KEYS):
        se = np.nan_to_num(resp[key + "_se"])
        out[k, 0] = n_groups
        out[k, 1] = resp[key]
        out[k, 2] = se * se * n_groups * max(n_groups - 1, 0)
    return out


def combine(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    na, ma, Ma = a[:, 0], a[:, 1], a[:, 2]
    nb, mb, Mb = b[:, 0], b[:, 1], b[:, 2]
    n = na + nb
    with np.errstate(invalid="ignore", divide="ignore"):
        d = mb - ma
        m = np.where(n > 0, ma + d * np.where(n > 0, nb / n, 0.0), 0.0)
        M2 = Ma + Mb + np.where(n > 0, d * d * na * nb / n, 0.0)
    return np.stack([n, m, M2], axis=1)


def from_moments(mom: np.ndarray, t: np.ndarray) -> dict:
    out = {"t": t}
    for k, key in enumerate(KEYS):
        n, m, M2 = mom[k]
        with np.errstate(invalid="ignore", divide="ignore"):
            se = np.sqrt(M2 / (n * (n - 1)))
        out[key] = m
        out[key + "_se"] = se
        out["n_groups"] = n
    return out


def merge_ranks(resp: dict, n_groups: int, group=None) -> dict:
    """All-gather every rank's moments and fold them in rank order."""
    import torch
    import torch.distributed as dist

    mom = to_moments(resp, n_groups)
    world = dist.get_world_size(group)
    t = torch.from_numpy(mom)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    acc = parts[0].cpu().numpy()
    for p in parts[1:]:
        acc = combine(acc, p.cpu().numpy())
    return from_moments(acc, resp["t"])
