"""Multi-rank merge of ensemble statistics: world_size-2 gloo ranks on CPU
split the oracle's mother groups; the merged responses equal the responses
of all groups reduced together."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2312_02990_gb300 import merge


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, B, Om, out_q, M=4):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    G = B.shape[0] // M
    lo, hi = (0, G // 2 + 1) if rank == 0 else (G // 2 + 1, G)   # uneven split
    r = oracle.responses(B[M * lo:M * hi], Om[M * lo:M * hi], M, 0.0025)
    m = merge.merge_ranks(r, hi - lo, r["omega_mean"])
    if rank == 0:
        out_q.put({k: np.asarray(v) for k, v in m.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_reduction():
    rng = np.random.default_rng(0)
    G, S = 9, 40
    B = rng.standard_normal((4 * G, S)).cumsum(axis=1) * 0.01
    Om = np.repeat(rng.standard_normal(G), 4) * np.tile([1, 1, -1, -1], G)
    full = oracle.responses(B, Om, 4, 0.0025)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, B, Om, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k in merge.KEYS:
        assert np.allclose(res[k], full[k], rtol=1e-12, atol=1e-15), k
        assert np.allclose(res[k + "_se"][1:], full[k + "_se"][1:], rtol=1e-10, atol=1e-15), k
    assert np.all(res["n_groups"] == G)


def test_combine_is_exact_for_known_moments():
    x = np.arange(10.0)
    a = merge.to_moments({"t": [0], "corr": [x[:3].mean()], "corr_se": [x[:3].std(ddof=1) / np.sqrt(3)],
                          "dav": [0.0], "dav_se": [0.0], "ttcf": [0.0], "ttcf_se": [0.0]}, 3)
    b = merge.to_moments({"t": [0], "corr": [x[3:].mean()], "corr_se": [x[3:].std(ddof=1) / np.sqrt(7)],
                          "dav": [0.0], "dav_se": [0.0], "ttcf": [0.0], "ttcf_se": [0.0]}, 7)
    m = merge.from_moments(merge.combine(a, b), np.array([0.0]))
    assert m["corr"][0] == pytest.approx(x.mean())
    assert m["corr_se"][0] == pytest.approx(x.std(ddof=1) / np.sqrt(10))


def test_two_rank_merge_keeps_the_eq4_form():
    """Two mappings per group (identity and time reversal: <Omega(0)> != 0),
    so the Eq. 4 form needs the global <Omega(0)>: the merged corrected
    response equals the corrected response of all groups reduced together,
    and differs from the plain one."""
    rng = np.random.default_rng(1)
    G, S, M = 11, 30, 2
    B = rng.standard_normal((M * G, S)).cumsum(axis=1) * 0.01 + 0.2
    Om = np.repeat(rng.standard_normal(G), M) + 0.3
    full_c = oracle.responses(B, Om, M, 0.0025, corrected=True)
    full = oracle.responses(B, Om, M, 0.0025)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, B, Om, q, M)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res["omega_mean"] == pytest.approx(Om.mean(), rel=1e-13)
    assert np.allclose(res["ttcf_c"], full_c["ttcf"], rtol=1e-12, atol=1e-15)
    assert np.allclose(res["ttcf"], full["ttcf"], rtol=1e-12, atol=1e-15)
    assert not np.allclose(res["ttcf_c"], res["ttcf"])
