"""GPU parity of the planar elongational daughters (TTCF_BULK_WCA_ELONG,
grad u = diag(eps, 0, -eps) in a deforming box) against the FP64 oracle,
through the C ABI.

Tolerances (stated per result):
  B(0), Omega(0)        relative 1e-12 (both sides IEEE double); the group
                        sums cancel exactly
  trajectories          FP64: positions, momenta, alpha 1e-9 and B(s) 1e-9
                        of max |B|; MIXED: B(s) 1e-4 of max |B| (double-float
                        state, FP32 pairs)
  affine crystal        closed-form lattice sums: FP64 1e-10, MIXED 1e-5 of
                        max |B| (FP32 pair distances)
  chunked runs          bitwise
  ensembles             within 2 combined standard errors
"""
import numpy as np
import pytest

import oracle
from elong_lattice import RC, fcc_vectors, lattice_sums
from paper_2312_02990_gb300 import inputs

pytestmark = pytest.mark.gpu

ELONG_MASK = 0x30003          # codes 0, 1, 16, 17
ELONG_SET = (0, 1, 16, 17)


@pytest.fixture(scope="module")
def ttcf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_02990_gb300 import ttcf as T
    T.load(build_if_missing=True)
    return T


def ctx(T, **kw):
    c = T.config_default()
    c.system = T.TTCF_BULK_WCA_ELONG
    c.mapping_mask = ELONG_MASK
    for k, v in kw.items():
        setattr(c, k, v)
    return T.Context(c)


def box_at(L, eps, t):
    return np.array([L[0] * np.exp(eps * t), L[1], L[2] * np.exp(-eps * t)])[:, None]


def test_spawn_gives_pxx_minus_pzz_and_cancels_omega(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    G = 8
    eps = np.geomspace(1e-1, 1e-6, G)
    with ctx(ttcf, precision=1, n_steps=4) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], eps, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 4 * G)
    for g in range(G):
        for k, m in enumerate(ELONG_SET):
            P = oracle.pressure(b, oracle.apply_mapping(b, m, ms[g], al[g])[0])[0]
            assert B[4 * g + k, 0] == pytest.approx(P[0] - P[2], rel=1e-12)
            assert Om[4 * g + k] == pytest.approx(-eps[g] * b.V * (P[0] - P[2]) / b.T, rel=1e-12)
        assert Om[4 * g:4 * g + 4].sum() == 0.0
        assert B[4 * g:4 * g + 4, 0].sum() == 0.0


@pytest.mark.parametrize("precision", [0, 1])
def test_daughters_follow_the_oracle(ttcf, eq_mothers_256, precision):
    """Two groups at eps = +0.2 and -0.1, 60 steps sampled every 2."""
    b, ms, al = eq_mothers_256
    rates = np.array([0.2, -0.1])
    n, se = 60, 2
    with ctx(ttcf, precision=precision, n_steps=n, sample_every=se, keep_state=1) as c:
        bid = c.spawn_daughters(ms[:2], al[:2], rates, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 8)
        states = [c.get_state(bid, d, b.n) for d in range(8)]
        stat = c.group_status(bid, 2)
    assert np.all(stat == 0)
    for d in range(8):
        g, k = divmod(d, 4)
        Bo, omo, fin, fa = oracle.daughter_elong(b, ms[g], al[g], ELONG_SET[k], rates[g], n,
                                                 sample_every=se)
        assert Om[d] == pytest.approx(omo, rel=1e-12)
        scale = np.abs(Bo).max()
        if precision == 0:
            assert np.abs(B[d] - Bo).max() < 1e-9 * scale, d
            s, a, delta = states[d]
            Lt = box_at(b.L, rates[g], n * b.dt)
            dx = s[:3] - fin[:3]
            dx -= Lt * np.rint(dx / Lt)
            assert np.abs(dx).max() < 1e-9, d
            assert np.abs(s[3:] - fin[3:]).max() < 1e-9, d
            assert a == pytest.approx(fa, abs=1e-9) and delta == 0.0
            assert np.all(s[:3] >= -0.5 * Lt) and np.all(s[:3] < 0.5 * Lt)
        else:
            assert np.abs(B[d] - Bo).max() < 1e-4 * scale, d


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_affine_crystal_follows_the_closed_form(ttcf, precision, tol):
    """A perfect FCC crystal at rest under eps = 0.5 for 300 steps: zero
    forces, affine positions, and P_xx - P_zz a lattice sum over the
    deformed neighbour shell (the compression brings it inside r_c)."""
    N, eps, n = 256, 0.5, 300
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))
    st = np.zeros((1, 6, N))
    st[0, :3] = inputs.fcc_lattice(N)
    with ctx(ttcf, precision=precision, n_steps=n, mapping_mask=1, keep_state=1) as c:
        bid = c.spawn_daughters(st, None, eps, box=b.L)
        c.run()
        B, _ = c.daughter_series(bid, 1)
        s, a, _ = c.get_state(bid, 0, N)
    R0 = fcc_vectors(b.L[0] / inputs.fcc_cells_for(N), 2.0 * RC)
    Bc = np.array([lattice_sums(R0, N, b.V, k * b.dt, eps)[0] for k in range(n + 1)])
    assert np.abs(Bc).max() > 1.0
    assert np.abs(B[0] - Bc).max() < tol * np.abs(Bc).max()
    assert a == pytest.approx(-b.dof * b.T * n * b.dt / b.Q, rel=1e-9)
    E = np.array([np.exp(eps * n * b.dt), 1.0, np.exp(-eps * n * b.dt)])[:, None]
    Lt = box_at(b.L, eps, n * b.dt)
    d = s[:3] - E * st[0, :3]
    d -= Lt * np.rint(d / Lt)
    assert np.abs(d).max() < (1e-10 if precision == 0 else 1e-5)


def test_two_cells_along_the_compressed_axis(ttcf):
    """N = 108 at eps = 0.5 for 400 steps: the z edge shrinks from 5.04 to
    3.06, so the list cells (at least r_c + skin wide) number two along z
    and the list build scans each of them once at the minimum image (FP64
    against the oracle, which takes every image there)."""
    N, eps, n = 108, 0.5, 400
    b = oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))
    ms, al = oracle.mother(b, inputs.initial_state(N, 3), 2000, 1, 10)
    assert b.L[2] * np.exp(-eps * n * b.dt) < 3 * RC
    with ctx(ttcf, precision=0, n_steps=n, keep_state=1) as c:
        bid = c.spawn_daughters(ms, al, eps, box=b.L)
        c.run()
        B, _ = c.daughter_series(bid, 4)
        states = [c.get_state(bid, d, N) for d in range(4)]
    for d in range(4):
        Bo, _, fin, _ = oracle.daughter_elong(b, ms[0], al[0], ELONG_SET[d], eps, n)
        assert np.abs(B[d] - Bo).max() < 1e-9 * np.abs(Bo).max(), d
        Lt = box_at(b.L, eps, n * b.dt)
        dx = states[d][0][:3] - fin[:3]
        dx -= Lt * np.rint(dx / Lt)
        assert np.abs(dx).max() < 1e-9, d


@pytest.mark.parametrize("precision", [0, 1])
def test_odd_atom_count(ttcf, precision):
    """N = 255 (one atom taken out of a 256-atom state): with an odd N the
    momentum slots end off a 16-byte boundary, which the shared-memory
    layout pads for the float4 and double arrays behind them."""
    N = 255
    L = tuple(inputs.bulk_box(256))
    b = oracle.Bulk(n=N, L=L)
    st = np.ascontiguousarray(inputs.jittered_states(256, 1, seed=23, amp=0.1)[:, :, 1:])
    eps, n = 0.1, 30
    with ctx(ttcf, precision=precision, n_steps=n) as c:
        bid = c.spawn_daughters(st, None, eps, box=b.L)
        c.run()
        B, _ = c.daughter_series(bid, 4)
        stat = c.group_status(bid, 1)
    assert np.all(stat == 0)
    for d in range(4):
        Bo = oracle.daughter_elong(b, st[0], 0.0, ELONG_SET[d], eps, n)[0]
        assert np.abs(B[d] - Bo).max() < (1e-9 if precision == 0 else 1e-4) * np.abs(Bo).max(), d


@pytest.mark.parametrize("precision", [0, 1])
def test_chunked_run_is_bitwise_equal(ttcf, eq_mothers_256, precision):
    b, ms, al = eq_mothers_256
    out = []
    for chunks in ((90,), (30, 45, 15)):
        with ctx(ttcf, precision=precision, n_steps=90, keep_state=1) as c:
            bid = c.spawn_daughters(ms[:3], al[:3], 0.05, box=b.L)
            for k in chunks:
                c.run(k)
            B, _ = c.daughter_series(bid, 12)
            s, a, _ = c.get_state(bid, 6, b.n)
            out.append((B, s, a))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


def test_mixed_ensemble_within_two_standard_errors(ttcf, eq_mothers_256):
    """48 mother states x 4 mappings, eps = 0.1, 300 steps: the TTCF and
    direct responses and the elongational viscosity against the oracle's
    ensemble on the same mothers."""
    b, ms, al = eq_mothers_256
    eps, n = 0.1, 300
    Bo, Omo = oracle.daughters_elong(b, ms, al, eps, n)
    ro = oracle.responses(Bo, Omo, 4, b.dt)
    with ctx(ttcf, precision=1, n_steps=n) as c:
        bid = c.spawn_daughters(ms, al, eps, box=b.L)
        c.run()
        r = c.response(bid)
        v = c.viscosity(bid)
        st = c.get_stats()
    assert st["rebuilds"] > 2 * 4 * len(ms)   # the lists were rebuilt along the way
    for k in ("dav", "ttcf"):
        for s in (100, 200, 300):
            se = np.hypot(r[k + "_se"][s], ro[k + "_se"][s])
            assert abs(r[k][s] - ro[k][s]) < 2.0 * se + 1e-12, (k, s)
    assert np.allclose(v["eta_ttcf"], -r["ttcf"] / (4 * eps), rtol=1e-12, atol=0)
    assert np.allclose(v["eta_ttcf_se"], r["ttcf_se"] / (4 * eps), rtol=1e-12, atol=0)


def test_rejects_a_rate_that_would_collapse_the_box(ttcf):
    """eps = 1 over 1000 steps would compress z from 6.72 to 0.55 < 2 r_c:
    ttcf_spawn_daughters refuses it before any work is queued."""
    N = 256
    st = inputs.jittered_states(N, 1, seed=2, amp=0.05)
    with ctx(ttcf, precision=1, n_steps=1000) as c:
        with pytest.raises(ttcf.TTCFError):
            c.spawn_daughters(st, None, 1.0, box=inputs.bulk_box(N))
        with pytest.raises(ttcf.TTCFError):
            c.spawn_daughters(st, None, -1.0, box=inputs.bulk_box(N))


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_continues_bitwise(ttcf, eq_mothers_256, tmp_path, precision):
    """An elongational run written to disk after 30 of 80 steps and continued
    in a new context (which recomputes the list bounds and skin from the
    saved box and rates) gives bitwise the uninterrupted series."""
    b, ms, al = eq_mothers_256
    rates = np.array([0.1, -0.05])
    kw = dict(precision=precision, n_steps=80)
    with ctx(ttcf, **kw) as c:
        bid = c.spawn_daughters(ms[:2], al[:2], rates, box=b.L)
        c.run()
        B_ref, Om_ref = c.daughter_series(bid, 8)
    path = str(tmp_path / "elong.ckpt")
    with ctx(ttcf, **kw) as c:
        c.spawn_daughters(ms[:2], al[:2], rates, box=b.L)
        c.run(30)
        c.save(path)
    with ctx(ttcf, **kw) as c:
        c.load(path)
        c.run()
        B, Om = c.daughter_series(0, 8)
    assert np.array_equal(B, B_ref) and np.array_equal(Om, Om_ref)
