"""Merge of per-rank TTCF ensemble statistics (multi-GPU, weak scaling).

Each rank reduces its own mother groups on its GPU (``ttcf_response``,
``ttcf_omega_mean``); the groups are independent, so the ensemble over all
ranks follows from each rank's per-sample valid-group count n, means and
standard errors of the group integrand Y_g, direct average D_g and TTCF
estimate J_g (Eq. 1, 2), and its <Omega(0)>.  Ranks exchange those (a few
arrays of S doubles) and fold them in rank order with the pairwise update of
Chan, Golub and LeVeque (1979):

    n = n_a + n_b,  d = m_b - m_a,  m = m_a + d n_b / n,
    M2 = M2_a + M2_b + d^2 n_a n_b / n,      with M2 = se^2 n (n - 1),

so the merged means and standard errors equal those of one run over all
groups (up to rounding), independently of the backend.  <Omega(0)> folds the
same way (weights n).  The Eq. 4 form of the merged ensemble is then formed
from the merged means as in the library's own reduction:

    corr_c(s) = corr(s) - <Omega(0)> dav(s),  ttcf_c(t) = dav(0) + int_0^t corr_c

(trapezoid on the sample grid); its standard error is the plain estimator's.
"""
from __future__ import annotations

import numpy as np

KEYS = ("corr", "dav", "ttcf")


def to_moments(resp: dict, n_groups: int, omega_mean: float = 0.0) -> np.ndarray:
    """[len(KEYS) + 1, 3, S] array: (n, mean, M2) per key, then the row
    (n, <Omega(0)>, 0) broadcast over samples."""
    S = len(resp["t"])
    out = np.zeros((len(KEYS) + 1, 3, S))
    for k, key in enumerate(KEYS):
        se = np.nan_to_num(resp[key + "_se"])
        out[k, 0] = n_groups
        out[k, 1] = resp[key]
        out[k, 2] = se * se * n_groups * max(n_groups - 1, 0)
    out[-1, 0] = n_groups
    out[-1, 1] = omega_mean
    return out


def combine(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    na, ma, Ma = a[:, 0], a[:, 1], a[:, 2]
    nb, mb, Mb = b[:, 0], b[:, 1], b[:, 2]
    n = na + nb
    with np.errstate(invalid="ignore", divide="ignore"):
        d = mb - ma
        m = np.where(n > 0, ma + d * np.where(n > 0, nb / n, 0.0), 0.0)
        M2 = Ma + Mb + np.where(n > 0, d * d * na * nb / n, 0.0)
    out = np.stack([n, m, M2], axis=1)
    out[-1, 2] = 0.0   # no spread is carried for <Omega(0)>
    return out


def from_moments(mom: np.ndarray, t: np.ndarray) -> dict:
    t = np.asarray(t, dtype=np.float64)
    out = {"t": t}
    for k, key in enumerate(KEYS):
        n, m, M2 = mom[k]
        with np.errstate(invalid="ignore", divide="ignore"):
            se = np.sqrt(M2 / (n * (n - 1)))
        out[key] = m
        out[key + "_se"] = se
        out["n_groups"] = n
    om = float(mom[-1, 1, 0])
    out["omega_mean"] = om
    ds = float(t[1] - t[0]) if t.size > 1 else 0.0
    corr_c = out["corr"] - om * out["dav"]
    ttcf_c = np.empty_like(corr_c)
    run = out["dav"][0]
    ttcf_c[0] = run
    for s in range(1, corr_c.size):
        run += 0.5 * ds * (corr_c[s - 1] + corr_c[s])
        ttcf_c[s] = run
    out["corr_c"] = corr_c
    out["ttcf_c"] = ttcf_c
    return out


def merge_ranks(resp: dict, n_groups: int, omega_mean: float = 0.0, group=None) -> dict:
    """All-gather every rank's moments and fold them in rank order."""
    import torch
    import torch.distributed as dist

    mom = to_moments(resp, n_groups, omega_mean)
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
