"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (stated per result):
  forces, FP64 mode     relative 1e-11 (summation order only)
  forces, MIXED mode    ||dF|| / ||F|| <= 1e-5 per state (spec bound);
                        per atom |dF_i| <= 2e-4 * F_rms (FP32 positions:
                        half an ulp of |x| <= L/2 moves a pair by ~2.4e-7,
                        and the WCA force changes by 13/r per unit r)
  B(0), Omega(0)        relative 1e-12 (both sides IEEE double)
  50-step trajectory    FP64: 1e-9; MIXED: positions 1e-6, momenta 1e-5
  ensembles             within 2 combined standard errors
"""
import numpy as np
import pytest

import oracle
from paper_2312_02990_gb300 import inputs

pytestmark = pytest.mark.gpu


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
    for k, v in kw.items():
        setattr(c, k, v)
    return T.Context(c)


def bulk(N):
    return oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)))


def min_image_diff(a, b, L):
    d = a - b
    return d - L * np.rint(d / L)


# ------------------------------------------------------------- forces ----
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [108, 256, 500, 2048])
def test_forces_match_oracle(ttcf, precision, N):
    b = bulk(N)
    st = inputs.jittered_states(N, 3, seed=100 + N, amp=0.1)
    rng = np.random.default_rng(N)
    deltas = [0.0, rng.uniform(-0.5, 0.5) * b.L[0], 0.5 * b.L[0] - 1e-3]
    with ctx(ttcf, precision=precision) as c:
        for k, delta in enumerate(deltas):
            F, W, U = c.forces(st[k], b.L, delta)
            Fo, Wo, Uo = oracle.forces(b, st[k], delta)
            err = np.linalg.norm(F[0] - Fo) / np.linalg.norm(Fo)
            frms = np.sqrt(np.mean(np.sum(Fo ** 2, axis=0)))
            per_atom = np.max(np.linalg.norm(F[0] - Fo, axis=0)) / frms
            if precision == 0:
                assert err < 1e-11 and per_atom < 1e-10
                assert W[0, 3] == pytest.approx(Wo[3], rel=1e-11)
            else:
                assert err < 1e-5, err
                assert per_atom < 2e-4, per_atom
                assert W[0, 3] == pytest.approx(Wo[3], rel=1e-5, abs=1e-5 * abs(Wo[:3]).max())
            assert U[0] == pytest.approx(Uo, rel=1e-11)
            assert np.all(W[0, [0, 1, 2, 4, 5]] == pytest.approx(Wo[[0, 1, 2, 4, 5]], rel=1e-11))


@pytest.mark.parametrize("precision", [0, 1])
def test_odd_atom_count(ttcf, precision):
    """N = 255 (one atom taken out of a 256-atom state): forces and a 30-step
    run against the oracle.  With an odd N the FP64 position arrays end off
    a 16-byte boundary, which the shared-memory layout pads for the float4
    arrays behind them."""
    N = 255
    L = tuple(inputs.bulk_box(256))
    b = oracle.Bulk(n=N, L=L)
    st = np.ascontiguousarray(inputs.jittered_states(256, 2, seed=17, amp=0.1)[:, :, 1:])
    with ctx(ttcf, precision=precision) as c:
        F, W, U = c.forces(st[0], b.L, 0.0)
    Fo, Wo, Uo = oracle.forces(b, st[0], 0.0)
    err = np.linalg.norm(F[0] - Fo) / np.linalg.norm(Fo)
    assert err < (1e-11 if precision == 0 else 1e-5), err
    assert U[0] == pytest.approx(Uo, rel=1e-11)
    gamma, n = 0.02, 30
    with ctx(ttcf, precision=precision, n_steps=n) as c:
        bid = c.spawn_daughters(st, None, gamma, box=b.L)
        c.run()
        B, _ = c.daughter_series(bid, 8)
        stat = c.group_status(bid, 2)
    assert np.all(stat == 0)
    for d in range(8):
        Bo = oracle.daughter(b, st[d // 4], 0.0, d % 4, gamma, n)[0]
        assert np.abs(B[d] - Bo).max() < (1e-10 if precision == 0 else 1e-4) * np.abs(Bo).max()


# -------------------------------------------------------------- spawn ----
def test_spawn_matches_oracle_and_cancels_exactly(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    G = 12
    gam = np.geomspace(1e-1, 1e-7, G)
    with ctx(ttcf, precision=1, n_steps=4, sample_every=1) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], gam, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 4 * G)
    for g in range(G):
        for m in range(4):
            mo, _ = oracle.apply_mapping(b, m, ms[g], al[g])
            P = oracle.pressure(b, mo)[0][3]
            assert B[4 * g + m, 0] == pytest.approx(P, rel=1e-12)
            assert Om[4 * g + m] == pytest.approx(-gam[g] * b.V * P / b.T, rel=1e-12)
        assert Om[4 * g:4 * g + 4].sum() == 0.0
        assert B[4 * g:4 * g + 4, 0].sum() == 0.0


# -------------------------------------------------------- trajectories ----
@pytest.mark.parametrize("precision,tol_x,tol_p", [(0, 1e-9, 1e-9), (1, 1e-6, 1e-5)])
def test_first_50_steps_follow_the_oracle(ttcf, eq_mothers_256, precision, tol_x, tol_p):
    b, ms, al = eq_mothers_256
    G, n, gamma = 3, 50, 0.05
    with ctx(ttcf, precision=precision, n_steps=n, keep_state=1) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], gamma, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 4 * G)
        L = np.asarray(b.L)[:, None]
        for g in range(G):
            for m in range(4):
                Bo, omo, fin, fa = oracle.daughter(b, ms[g], al[g], m, gamma, n)
                s, a, d = c.get_state(bid, 4 * g + m, b.n)
                dx = min_image_diff(s[:3], fin[:3], L)
                assert np.abs(dx).max() < tol_x
                assert np.abs(s[3:] - fin[3:]).max() < tol_p
                assert a == pytest.approx(fa, abs=tol_p)
                scale = np.abs(Bo).max()
                assert np.abs(B[4 * g + m] - Bo).max() < (1e-10 if precision == 0 else 1e-4) * scale


def test_fp64_active_lists_under_strong_shear_follow_the_oracle(ttcf, eq_mothers_256):
    """FP64 force passes walk each atom's active list (the Verlet entries
    within r_c + 0.1 sigma, refreshed from the sorted Verlet list when an
    atom's path length or the Lees-Edwards offset could close the gap).  At
    gamma = 1 the offset alone forces a refresh every few steps and the
    Verlet lists are rebuilt often: 300 steps of 8 daughters against the
    oracle, positions and momenta to 1e-9."""
    b, ms, al = eq_mothers_256
    G, n, gamma = 2, 300, 1.0
    with ctx(ttcf, precision=0, n_steps=n, keep_state=1) as c:
        bid = c.spawn_daughters(ms[:G], al[:G], gamma, box=b.L)
        c.run()
        st = c.get_stats()
        B, _ = c.daughter_series(bid, 4 * G)
        states = [c.get_state(bid, d, b.n) for d in range(4 * G)]
    assert st["rebuilds"] > 4 * G * 3
    Lx, Ly, Lz = b.L
    for d in range(4 * G):
        Bo, _, fin, fa = oracle.daughter(b, ms[d // 4], al[d // 4], d % 4, gamma, n)
        s, a, delta = states[d]
        # Lees-Edwards minimum image: a y image carries the x offset delta
        dx, dy, dz = s[:3] - fin[:3]
        ny = np.rint(dy / Ly)
        dy, dx = dy - ny * Ly, dx - ny * delta
        dx -= Lx * np.rint(dx / Lx)
        dz -= Lz * np.rint(dz / Lz)
        assert max(np.abs(dx).max(), np.abs(dy).max(), np.abs(dz).max()) < 1e-9, d
        assert np.abs(s[3:] - fin[3:]).max() < 1e-9, d
        assert a == pytest.approx(fa, abs=1e-9)
        assert np.abs(B[d] - Bo).max() < 1e-9 * np.abs(Bo).max(), d


def test_config1_fp64_ensemble_matches_oracle(ttcf):
    """N=256, 10 mother states 200 steps apart, x4 mappings, 500 steps at
    gamma = 1e-3, FP64 (the smallest configuration, in full)."""
    N = 256
    b = bulk(N)
    ms, al = oracle.mother(b, inputs.initial_state(N, inputs.BASE_SEED), n_eq=4000,
                           n_states=10, spacing=200)
    gamma, n = 1e-3, 500
    Bo, Omo = oracle.daughters(b, ms, al, gamma, n)
    ro = oracle.responses(Bo, Omo, 4, b.dt)
    with ctx(ttcf, precision=0, n_steps=n) as c:
        bid = c.spawn_daughters(ms, al, gamma, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 40)
        r = c.response(bid)
        v = c.viscosity(bid)
    # FP64 on both sides: chaos amplifies summation-order rounding only
    assert np.abs(Om - Omo).max() <= 1e-12 * np.abs(Omo).max()
    assert np.abs(B - Bo).max() < 1e-6 * np.abs(Bo).max()
    for k in ("corr", "dav", "ttcf"):
        assert np.allclose(r[k], ro[k], rtol=1e-5, atol=1e-6 * np.abs(ro[k]).max()), k
        assert np.allclose(r[k + "_se"][1:], ro[k + "_se"][1:], rtol=1e-3, atol=1e-9), k
    assert r["dav_se"][0] == 0.0 and r["dav"][0] == 0.0
    assert np.allclose(v["eta_ttcf"], -ro["ttcf"] / gamma, rtol=1e-5, atol=1e-5)


def test_mixed_ensemble_within_two_standard_errors(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    gamma, n = 0.1, 300
    Bo, Omo = oracle.daughters(b, ms, al, gamma, n)
    ro = oracle.responses(Bo, Omo, 4, b.dt)
    with ctx(ttcf, precision=1, n_steps=n) as c:
        bid = c.spawn_daughters(ms, al, gamma, box=b.L)
        c.run()
        r = c.response(bid)
    for k in ("dav", "ttcf"):
        for s in (100, 200, 300):
            se = np.hypot(r[k + "_se"][s], ro[k + "_se"][s])
            assert abs(r[k][s] - ro[k][s]) < 2.0 * se + 1e-12, (k, s)


def test_chunked_run_is_bitwise_equal_and_deterministic(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    out = []
    for chunks in ((130,), (40, 64, 26), (130,)):
        with ctx(ttcf, precision=1, n_steps=130, keep_state=1) as c:
            bid = c.spawn_daughters(ms[:4], al[:4], 0.01, box=b.L)
            for k in chunks:
                c.run(k)
            B, Om = c.daughter_series(bid, 16)
            s, a, d = c.get_state(bid, 5, b.n)
            out.append((B, s, a))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0])
        assert np.array_equal(o[1], out[0][1]) and o[2] == out[0][2]


def test_gpu_mothers_are_equilibrium_samples(ttcf):
    """Mother states from the GPU sampler: FP64 mode follows the oracle's
    mother for 50 steps; MIXED mothers reach the same temperature and
    potential energy (the NVT target T = 0.722 at rho = 0.8442)."""
    N = 256
    b = bulk(N)
    s0 = inputs.initial_state(N, 5)
    with ctx(ttcf, precision=0) as c:
        g, ga = c.sample_mothers(s0, b.L, n_eq=0, n_states=1, spacing=50)
    o, oa = oracle.mother(b, s0, n_eq=0, n_states=1, spacing=50)
    L = np.asarray(b.L)[:, None]
    assert np.abs(min_image_diff(g[0, 0, :3], o[0, :3], L)).max() < 1e-9
    assert np.abs(g[0, 0, 3:] - o[0, 3:]).max() < 1e-9
    assert ga[0, 0] == pytest.approx(oa[0], abs=1e-9)
    with ctx(ttcf, precision=1) as c:
        g, ga = c.sample_mothers(np.stack([inputs.initial_state(N, 10 + k) for k in range(8)]),
                                 b.L, n_eq=4000, n_states=8, spacing=200)
    states = g.reshape(-1, 6, N)
    T = np.mean([np.sum(s[3:] ** 2) / (3 * N) for s in states])
    U = np.mean([oracle.pressure(b, s)[1] / N for s in states])
    Uo = np.mean([oracle.pressure(b, s)[1] / N for s in
                  oracle.mother(b, inputs.initial_state(N, 99), 4000, 16, 200)[0]])
    assert T == pytest.approx(0.722, rel=0.03)
    assert U == pytest.approx(Uo, rel=0.05)


# ------------------------------------------------------------ edge cases --
def test_subset_of_mappings_uses_eq4_correction(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    gamma, n = 0.05, 60
    with ctx(ttcf, precision=0, n_steps=n, mapping_mask=0x3) as c:   # no x-reflections
        bid = c.spawn_daughters(ms[:8], al[:8], gamma, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 16)
        r = c.response(bid, corrected=True)
    Bo, Omo = oracle.daughters(b, ms[:8], al[:8], gamma, n, mapping_mask=0x3)
    ro = oracle.responses(Bo, Omo, 2, b.dt, corrected=True)
    assert abs(Omo.sum()) > 1e-3 * np.abs(Omo).sum()   # <Omega(0)> != 0 without x-reflections
    assert np.allclose(r["ttcf"], ro["ttcf"], rtol=1e-6, atol=1e-9)
    # with corrected=1 the integrand is the Eq. 4 form
    corr_c = ro["corr"] - ro["omega_mean"] * ro["dav"]
    assert np.allclose(r["corr"], corr_c, rtol=1e-6, atol=1e-9)


def test_zero_field_and_reset_alpha(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    with ctx(ttcf, precision=0, n_steps=40, reset_alpha=1, keep_state=1) as c:
        bid = c.spawn_daughters(ms[:2], al[:2], 0.0, box=b.L)
        c.run()
        B, Om = c.daughter_series(bid, 8)
        s, a, _ = c.get_state(bid, 1, b.n)
    assert np.all(Om == 0.0)
    Bo, _, fin, fa = oracle.daughter(b, ms[0], al[0], 1, 0.0, 40, reset_alpha=True)
    assert np.allclose(B[1], Bo, rtol=1e-9, atol=1e-12)
    assert a == pytest.approx(fa, abs=1e-9)


def test_ragged_sizes_and_uneven_batch_in_one_run(ttcf):
    """Batches of N = 108, 256, 500 and 864 with different shear rates run
    together (one persistent launch per size class); each daughter matches
    the oracle for its first 30 steps."""
    with ctx(ttcf, precision=0, n_steps=30) as c:
        ids, refs = [], []
        for N, gam in ((108, 1e-2), (256, 1e-4), (500, 1e-3), (864, 1e-6)):
            b = bulk(N)
            st = inputs.jittered_states(N, 2, seed=N, amp=0.05)
            ids.append(c.spawn_daughters(st, np.array([0.1, -0.2]), gam, box=b.L))
            refs.append((b, st, gam))
        c.run()
        for bid, (b, st, gam) in zip(ids, refs):
            B, Om = c.daughter_series(bid, 8)
            for g in range(2):
                for m in range(4):
                    Bo, omo, _, _ = oracle.daughter(b, st[g], [0.1, -0.2][g], m, gam, 30)
                    assert np.allclose(B[4 * g + m], Bo, rtol=1e-8, atol=1e-10 * np.abs(Bo).max())
                    assert Om[4 * g + m] == pytest.approx(omo, rel=1e-12, abs=1e-300)


def test_uneven_batch_in_one_graph_launch(ttcf):
    """The uneven-batch workload at its sizes: N = 256, 864 and 4000 mixed
    with shear rates 1e-2 ... 1e-6 in one graph-captured run (MIXED), launch
    shapes chosen by the autotuner per N (N = 4000 takes the index-only list
    layout); two daughters of every (N, rate) batch against the oracle for
    100 steps."""
    sizes, rates, n = (256, 864, 4000), [1e-2, 1e-3, 1e-4, 1e-5, 1e-6], 100
    states = {N: inputs.jittered_states(N, 2, seed=500 + N, amp=0.05) for N in sizes}
    with ctx(ttcf, precision=1, n_steps=n, use_graph=1) as c:
        for N in sizes:
            c.autotune(states[N], bulk(N).L, n_steps=20)
        ids = {(N, g): c.spawn_daughters(states[N], None, g, box=bulk(N).L) for N in sizes for g in rates}
        c.run()
        out = {k: c.daughter_series(b, 8) for k, b in ids.items()}
        status = {k: c.group_status(b, 2) for k, b in ids.items()}
    for (N, g), (B, Om) in out.items():
        assert np.all(status[(N, g)] == 0), (N, g)
        b = bulk(N)
        for d in (0, 5):   # group 0 unmapped, group 1 time-reversed
            Bo, omo, _, _ = oracle.daughter(b, states[N][d // 4], 0.0, d % 4, g, n)
            assert Om[d] == pytest.approx(omo, rel=1e-10, abs=1e-300)
            assert np.abs(B[d] - Bo).max() < 1e-4 * np.abs(Bo).max(), (N, g, d)


def test_invalid_inputs_are_rejected(ttcf):
    T = ttcf
    with ctx(T, precision=1, n_steps=10) as c:
        with pytest.raises(T.TTCFError) as e:
            c.run()
        assert e.value.status == T.TTCF_E_STATE
        b = bulk(256)
        st = inputs.jittered_states(256, 1, seed=1)
        with pytest.raises(T.TTCFError) as e:   # box too small for the cell search
            c.spawn_daughters(st, None, 0.1, box=(3.0, 3.0, 3.0))
        assert e.value.status == T.TTCF_E_INVALID
        with pytest.raises(T.TTCFError) as e:
            c.spawn_daughters(np.zeros((1, 6, 5000)), None, 0.1, box=(20.0, 20.0, 20.0))
        assert e.value.status == T.TTCF_E_INVALID
        with pytest.raises(T.TTCFError):
            c.spawn_daughters(st, None, np.nan, box=b.L)
        bid = c.spawn_daughters(st, None, 0.1, box=b.L)
        with pytest.raises(T.TTCFError) as e:
            c.response(bid)
        assert e.value.status == T.TTCF_E_STATE


def test_overlapping_atoms_are_reported_not_crashed(ttcf, eq_mothers_256):
    """A mother with two atoms almost on top of each other blows up; its
    group is flagged and excluded, the other groups are unaffected."""
    T = ttcf
    b, ms, al = eq_mothers_256
    bad = ms[:3].copy()
    bad[1, :3, 7] = bad[1, :3, 8] + 1e-3
    with ctx(T, precision=1, n_steps=50) as c:
        bid = c.spawn_daughters(bad, al[:3], 0.01, box=b.L)
        assert c.run(allow_numeric=True) == T.TTCF_E_NUMERIC
        st = c.group_status(bid, 3)
        r = c.response(bid)
    assert st[0] == 0 and st[2] == 0 and st[1] != 0
    assert np.all(np.isfinite(r["ttcf"])) and np.all(np.isfinite(r["dav"]))


def test_timeout_aborts_and_context_stays_usable(ttcf, eq_mothers_256):
    T = ttcf
    b, ms, al = eq_mothers_256
    with ctx(T, precision=0, n_steps=200000, timeout_s=0.5) as c:
        bid = c.spawn_daughters(ms[:2], al[:2], 0.01, box=b.L)
        with pytest.raises(T.TTCFError) as e:
            c.run()
        assert e.value.status == T.TTCF_E_TIMEOUT
        assert np.all(c.group_status(bid, 2) & T.D_ABORTED)
    with ctx(T, precision=1, n_steps=20) as c:   # the device is still usable
        bid = c.spawn_daughters(ms[:1], al[:1], 0.01, box=b.L)
        c.run()


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (0, 1e-9)])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6])
def test_every_launch_variant_follows_the_oracle(ttcf, variant, precision, tol):
    """Each launch shape (atoms per thread, block size, register budget)
    gives the same 30-step trajectory responses as the oracle (N = 500, so
    that every variant is exercised with a ragged tail), in both precisions
    (the FP64 passes walk their active lists)."""
    N = 500
    b = bulk(N)
    st = inputs.jittered_states(N, 2, seed=9, amp=0.05)
    apt, maxt = [(1, 256), (2, 512), (2, 1024), (4, 512), (4, 512), (8, 512)][variant - 1]
    if apt * maxt < N:
        pytest.skip("variant cannot hold N")
    with ctx(ttcf, precision=precision, n_steps=30, kernel_variant=variant) as c:
        bid = c.spawn_daughters(st, None, 0.02, box=b.L)
        c.run()
        B, _ = c.daughter_series(bid, 8)
    for d in range(8):
        Bo, _, _, _ = oracle.daughter(b, st[d // 4], 0.0, d % 4, 0.02, 30)
        assert np.abs(B[d] - Bo).max() < tol * np.abs(Bo).max()


def test_autotuner_choice_is_used_and_exact(ttcf, eq_mothers_256):
    b, ms, al = eq_mothers_256
    with ctx(ttcf, precision=1, n_steps=40, keep_state=1) as c:
        v, skin, frac, t = c.autotune(ms[:4], b.L, shear_rate=1e-3, n_steps=20)
        assert 1 <= v <= 6 and skin in (0.3, 0.35, 0.4, 0.5, 0.6) and t > 0
        assert frac in (0.5, 2.0 / 3.0, 1.0)
        bid = c.spawn_daughters(ms[:2], al[:2], 1e-3, box=b.L)
        c.run()
        assert c.get_stats()["skin"] == skin
        s, a, _ = c.get_state(bid, 3, b.n)
    _, _, fin, fa = oracle.daughter(b, ms[0], al[0], 3, 1e-3, 40)
    L = np.asarray(b.L)[:, None]
    assert np.abs(min_image_diff(s[:3], fin[:3], L)).max() < 1e-6


def test_graph_and_stream_launches_agree_bitwise(ttcf):
    """One CUDA graph per run (persistent launches of two size classes on
    forked streams plus the reductions) gives the same bits as plain
    stream launches."""
    out = []
    for use_graph in (1, 0):
        with ctx(ttcf, precision=1, n_steps=50, use_graph=use_graph) as c:
            ids = []
            for N in (256, 864):
                b = bulk(N)
                ids.append((c.spawn_daughters(inputs.jittered_states(N, 3, seed=N, amp=0.05), None,
                                              1e-3, box=b.L), N))
            c.run()
            out.append([c.daughter_series(i, 12)[0] for i, _ in ids] + [c.response(i)["ttcf"] for i, _ in ids])
            assert c.get_stats()["launches"] == 2 + 3 * 2
    for a, b_ in zip(out[0], out[1]):
        assert np.array_equal(a, b_)
