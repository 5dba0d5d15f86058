"""GPU parity of the confined system (Example 2: Eq. 9, 10, 11) through the
C ABI against the FP64 oracle (oracle/confined.py) on the same inputs.

Tolerances (stated per result):
  Omega(0), wall forces at t = 0   relative 1e-10 (both sides IEEE double,
                                   different summation order)
  slab sums of p_x at t = 0        absolute 1e-9 (the device sums exact
                                   fixed point with 2^-40 resolution)
  slab counts                      exact at t = 0
  trajectories (MIXED, <= 40 steps) wall forces within 5e-4 of the series'
                                   RMS (FP32 pair forces: ~1e-5 expected);
                                   slab profiles: the MIXED positions differ
                                   from FP64 by up to ~1e-6, so an atom that
                                   close to a slab boundary may sit on either
                                   side (about one such atom per test); the
                                   total count is exact, at most a few atoms
                                   change slab, and every slab whose count
                                   agrees has its p_x sum within 5e-4
  mother states (30 steps)         positions 1e-6, momenta 5e-5 (30 steps of
                                   h = 0.005 with FP32 LJ forces whose error
                                   reaches ~1e-4 per atom), alpha 1e-6
  ensembles                        within 2 combined standard errors
"""
import numpy as np
import pytest

from oracle import confined as oc
from oracle import reduce as orr
from paper_2312_02990_gb300 import inputs

pytestmark = pytest.mark.gpu

NOBS = oc.N_OBS       # 2 wall stresses, 40 slab momenta, 40 slab counts, 2 inner wall layers
H = 10.0     # channel width: v = gamma h / 2


@pytest.fixture(scope="module")
def ttcf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_02990_gb300 import ttcf as T
    T.load(build_if_missing=True)
    return T


@pytest.fixture(scope="module")
def chan():
    """A small channel (10 x 10 rows, 2 wall layers) thermalised at rest by
    the oracle: 4 mother states 100 steps apart."""
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=3)
    sy = oc.Confined(types=s["types"], box=tuple(s["box"]))
    ms, al = oc.mother(sy, s["state"], s["lattice"], n_eq=1000, n_states=4, spacing=100)
    return s, sy, ms, al


def cctx(T, **kw):
    c = T.config_default()
    c.system = T.TTCF_CONFINED_LJ
    c.precision = T.TTCF_MIXED
    c.dt, c.T, c.tau_T = 0.005, 1.0, 0.25
    for k, v in kw.items():
        setattr(c, k, v)
    return T.Context(c)


def assert_profiles_close(Bg, Bo, n_fluid, max_moves=6):
    """Bg, Bo [NOBS, S] of one daughter (device, oracle)."""
    ns = oc.N_SLAB
    cg, co = Bg[2 + ns:2 + 2 * ns], Bo[2 + ns:2 + 2 * ns]
    assert np.all(cg.sum(axis=0) == n_fluid) and np.all(co.sum(axis=0) == n_fluid)
    dc = cg - co
    assert np.abs(dc).sum() <= 2 * max_moves, np.argwhere(dc != 0)
    same = dc == 0
    dp = np.abs(Bg[2:2 + ns] - Bo[2:2 + ns])
    assert dp[same].max() < 5e-4, dp[same].max()
    # the total fluid momentum does not depend on the slab assignment
    assert np.abs(Bg[2:2 + ns].sum(axis=0) - Bo[2:2 + ns].sum(axis=0)).max() < 5e-3
    # the p_x sums of the innermost wall layers
    assert np.abs(Bg[2 + 2 * ns:] - Bo[2 + 2 * ns:]).max() < 1e-3


def oracle_daughters(sy, ms, lat, al, gamma, n_steps, sample_every=1):
    """[D, NOBS, S] and Omega [D], d = 4 g + m."""
    sys2 = oc.Confined(types=sy.types, box=sy.box, vwall=gamma * H / 2)
    B, Om = oc.daughters(sys2, ms, lat, al, n_steps, sample_every)
    return np.ascontiguousarray(B.transpose(0, 2, 1)), Om


# -------------------------------------------------------------- spawn ----
def test_spawn_matches_oracle_and_cancels_exactly(ttcf, chan):
    s, sy, ms, al = chan
    G = ms.shape[0]
    gam = np.array([0.1, 1e-3, 1e-8, 0.05])
    with cctx(ttcf, n_steps=1) as c:
        bid = c.spawn_confined(ms, s["types"], s["lattice"], sy.box, al, gam)
        Bg, Om = c.daughter_series(bid, 4 * G, NOBS)
    for g in range(G):
        sys2 = oc.Confined(types=sy.types, box=sy.box, vwall=gam[g] * H / 2)
        for m in range(4):
            d = 4 * g + m
            Bo, omo, _ = oc.daughter(sys2, ms[g], s["lattice"], al[g], m, 0)
            assert Om[d] == pytest.approx(omo, rel=1e-10, abs=1e-12 * abs(omo) + 1e-300)
            assert Bg[d, :2, 0] == pytest.approx(Bo[0, :2], rel=1e-10, abs=1e-12)
            assert np.abs(Bg[d, 2:2 + oc.N_SLAB, 0] - Bo[0, 2:2 + oc.N_SLAB]).max() < 1e-9
            assert np.array_equal(Bg[d, 2 + oc.N_SLAB:2 + 2 * oc.N_SLAB, 0], Bo[0, 2 + oc.N_SLAB:2 + 2 * oc.N_SLAB])
            assert np.abs(Bg[d, 2 + 2 * oc.N_SLAB:, 0] - Bo[0, 2 + 2 * oc.N_SLAB:]).max() < 1e-9
        # Eq. 3: the four mappings cancel Omega(0), the wall forces and the
        # slab momenta exactly within each group
        grp = slice(4 * g, 4 * g + 4)
        assert Om[grp].sum() == 0.0
        assert np.all(Bg[grp, :2 + oc.N_SLAB, 0].sum(axis=0) == 0.0)
        assert np.all(Bg[grp, 2 + 2 * oc.N_SLAB:, 0].sum(axis=0) == 0.0)


# -------------------------------------------------------- trajectories ---
@pytest.mark.parametrize("gamma", [0.05, 1e-6])
def test_daughters_follow_oracle(ttcf, chan, gamma):
    s, sy, ms, al = chan
    n = 40
    with cctx(ttcf, n_steps=n) as c:
        bid = c.spawn_confined(ms[:1], s["types"], s["lattice"], sy.box, al[:1], gamma)
        c.run()
        Bg, Om = c.daughter_series(bid, 4, NOBS)
        st = c.group_status(bid, 1)
    assert st[0] == 0
    Bo, Omo = oracle_daughters(sy, ms[:1], s["lattice"], al[:1], gamma, n)
    assert Om == pytest.approx(Omo, rel=1e-10, abs=1e-300)
    for d in range(4):
        for w in (0, 1):
            rms = np.sqrt(np.mean(Bo[d, w] ** 2))
            dev = np.abs(Bg[d, w] - Bo[d, w]).max() / rms
            assert dev < 5e-4, (d, w, dev)
        assert_profiles_close(Bg[d], Bo[d], int(np.sum(s["types"] == 0)))


def test_walls_held_by_tethers_alone(ttcf, chan):
    """Wall-wall pairs switched off on both sides (the reading in which only
    the tethers hold the walls)."""
    s, sy, ms, al = chan
    n, g = 30, 0.05
    p = ttcf.confined_params_default()
    p.ww_on = 0
    with cctx(ttcf, n_steps=n) as c:
        bid = c.spawn_confined(ms[:1], s["types"], s["lattice"], sy.box, al[:1], g, params=p)
        c.run()
        Bg, Om = c.daughter_series(bid, 4, NOBS)
    sys2 = oc.Confined(types=sy.types, box=sy.box, vwall=g * H / 2, ww_on=False)
    Bo, Omo = oc.daughters(sys2, ms[:1], s["lattice"], al[:1], n, 1)
    Bo = Bo.transpose(0, 2, 1)
    for d in range(4):
        for w in (0, 1):
            rms = np.sqrt(np.mean(Bo[d, w] ** 2))
            assert np.abs(Bg[d, w] - Bo[d, w]).max() < 5e-4 * rms
        assert_profiles_close(Bg[d], Bo[d], int(np.sum(s["types"] == 0)))


def test_full_size_channel_short_run(ttcf):
    """The Example 2 geometry (10248 atoms, one daughter per CTA at the shared
    memory limit) from the generator's initial state, 20 steps."""
    s = inputs.confined_system()
    sy = oc.Confined(types=s["types"], box=tuple(s["box"]))
    ms = s["state"][None]
    al = np.zeros(1)
    gamma, n = 0.1, 20
    with cctx(ttcf, n_steps=n, sample_every=5) as c:
        bid = c.spawn_confined(ms, s["types"], s["lattice"], sy.box, al, gamma)
        c.run()
        Bg, Om = c.daughter_series(bid, 4, NOBS)
        st = c.group_status(bid, 1)
    assert st[0] == 0
    Bo, Omo = oracle_daughters(sy, ms, s["lattice"], al, gamma, n, 5)
    assert Om == pytest.approx(Omo, rel=1e-10, abs=1e-300)
    for d in range(4):
        for w in (0, 1):
            rms = np.sqrt(np.mean(Bo[d, w] ** 2))
            assert np.abs(Bg[d, w] - Bo[d, w]).max() < 5e-4 * rms
        assert_profiles_close(Bg[d], Bo[d], s["n_fluid"])


def test_odd_cell_count(ttcf):
    """A channel whose list grid has an odd number of cells (9 x 9 x 7): the
    shared-memory regions after the cell counts must stay 8-byte aligned."""
    s = inputs.confined_system(nx=11, nz=10, layers=2, seed=5)
    sy = oc.Confined(types=s["types"], box=tuple(s["box"]))
    ms, al = s["state"][None], np.zeros(1)
    with cctx(ttcf, n_steps=30, skin=0.4) as c:
        bid = c.spawn_confined(ms, s["types"], s["lattice"], sy.box, al, 0.02)
        c.run()
        Bg, Om = c.daughter_series(bid, 4, NOBS)
    Bo, Omo = oracle_daughters(sy, ms, s["lattice"], al, 0.02, 30)
    for d in range(4):
        for w in (0, 1):
            rms = np.sqrt(np.mean(Bo[d, w] ** 2))
            assert np.abs(Bg[d, w] - Bo[d, w]).max() < 5e-4 * rms
        assert_profiles_close(Bg[d], Bo[d], s["n_fluid"])


def test_escaped_atom_is_reported(ttcf, chan):
    """A fluid atom far behind a wall (|y| > Ly) flags its group
    TTCF_D_ESCAPED at the first list build; the other groups are unaffected
    and the reduction excludes the flagged one."""
    s, sy, ms, al = chan
    bad = ms[:2].copy()
    f = np.nonzero(s["types"] == 0)[0][0]
    bad[1, 1, f] = -1.2 * sy.box[1]
    with cctx(ttcf, n_steps=20) as c:
        bid = c.spawn_confined(bad, s["types"], s["lattice"], sy.box, al[:2], 0.01)
        st = c.run(allow_numeric=True)
        gs = c.group_status(bid, 2)
        r = c.response_obs(bid, 0)
    assert st == ttcf.TTCF_E_NUMERIC
    assert gs[0] == 0 and gs[1] & ttcf.D_ESCAPED
    assert np.all(np.isfinite(r["ttcf"]))


def test_zero_field_has_zero_dissipation(ttcf, chan):
    s, sy, ms, al = chan
    with cctx(ttcf, n_steps=20) as c:
        bid = c.spawn_confined(ms[:2], s["types"], s["lattice"], sy.box, al[:2], 0.0)
        c.run()
        B, Om = c.daughter_series(bid, 8, NOBS)
        r = c.response_obs(bid, 0)
    assert np.all(Om == 0.0)
    assert np.all(r["corr"] == 0.0)
    assert np.all(r["ttcf"] == r["ttcf"][0])


# ------------------------------------------------------------ mothers ----
def test_mother_sampling_matches_oracle(ttcf, chan):
    s, sy, ms, al = chan
    with cctx(ttcf) as c:
        out, oa = c.sample_mothers_confined(ms[0], s["types"], s["lattice"], sy.box, n_eq=10,
                                            n_states=2, spacing=10)
    ref, ra = oc.mother(sy, ms[0], s["lattice"], n_eq=10, n_states=2, spacing=10)
    L = np.array(sy.box)
    for k in range(2):
        for r in range(3):
            d = out[0, k, r] - ref[k, r]
            if r != 1:
                d -= L[r] * np.rint(d / L[r])
            assert np.abs(d).max() < 1e-6, (k, r)
        assert np.abs(out[0, k, 3:] - ref[k, 3:]).max() < 5e-5
        assert oa[0, k] == pytest.approx(ra[k], rel=1e-6, abs=1e-9)
        # x and z wrapped into the box
        assert np.all(np.abs(out[0, k, [0, 2]]) <= 0.5 * L[[0, 2], None] + 1e-9)


# ----------------------------------------------------------- ensembles ---
def test_ensemble_responses_match_oracle(ttcf, chan):
    s, sy, ms, al = chan
    gamma, n, se = 0.05, 200, 2
    G = ms.shape[0]
    with cctx(ttcf, n_steps=n, sample_every=se) as c:
        bid = c.spawn_confined(ms, s["types"], s["lattice"], sy.box, al, gamma)
        c.run()
        Bg, Om = c.daughter_series(bid, 4 * G, NOBS)
        got = {o: c.response_obs(bid, o) for o in (0, 1, 2 + 20, 2 + oc.N_SLAB + 20)}
    ds = se * 0.005
    Bo, Omo = oracle_daughters(sy, ms, s["lattice"], al, gamma, n, se)
    for o, r in got.items():
        # the device reduction of the device series: the oracle's formulas
        own = orr.responses(Bg[:, o], Om, 4, ds)
        for k in ("corr", "dav", "ttcf"):
            assert r[k] == pytest.approx(own[k], rel=1e-10, abs=1e-12 * (np.abs(own[k]).max() + 1e-300))
        # against the oracle's own daughters
        ref = orr.responses(Bo[:, o], Omo, 4, ds)
        tol = 2 * np.sqrt(r["ttcf_se"] ** 2 + ref["ttcf_se"] ** 2) + 1e-9
        assert np.all(np.abs(r["ttcf"] - ref["ttcf"]) <= tol)


def test_friction_matches_the_oracle_formula(ttcf, chan):
    """Eq. 12 from the device responses: slip velocity (innermost wall layer
    minus outermost fluid layer) and friction at both walls against
    oracle/reduce.friction on the same responses."""
    s, sy, ms, al = chan
    g = 0.05
    with cctx(ttcf, n_steps=100, sample_every=5) as c:
        bid = c.spawn_confined(ms, s["types"], s["lattice"], sy.box, al, g)
        c.run()
        resp = {o: c.response_obs(bid, o) for o in range(NOBS)}
        got = [c.friction(bid, w) for w in (0, 1)]
        with pytest.raises(ttcf.TTCFError):
            c.friction(bid, 2)
    for w in (0, 1):
        for est, key in (("ttcf", "ttcf"), ("dav", "dav")):
            n_layer = len(oc.inner_layer(s["types"], s["lattice"], w))
            assert n_layer == 100   # one FCC(111) layer of the 10 x 10 rows
            ref = orr.friction(resp, sy.box[1], H, w, n_layer, estimator=key)
            assert np.allclose(got[w]["slip_" + est], ref["slip"], rtol=1e-12, atol=1e-15)
            ok = np.isfinite(ref["xi"])
            assert np.allclose(got[w]["xi_" + est][ok], ref["xi"][ok], rtol=1e-10)
        # at t = 0 the four mappings cancel every p_x sum: no slip
        assert got[w]["slip_dav"][0] == 0.0


# ------------------------------------------------------------- errors ----
def test_invalid_inputs_are_rejected(ttcf, chan):
    T = ttcf
    s, sy, ms, al = chan
    c0 = T.config_default()
    c0.system = T.TTCF_CONFINED_LJ
    c0.precision = T.TTCF_FP64
    with pytest.raises(T.TTCFError):
        T.Context(c0)
    with T.Context() as c:   # a bulk context
        with pytest.raises(T.TTCFError) as e:
            c.spawn_confined(ms[:1], s["types"], s["lattice"], sy.box, al[:1], 0.1)
        assert e.value.status == T.TTCF_E_INVALID
    with cctx(T, n_steps=10) as c:
        with pytest.raises(T.TTCFError):
            c.spawn_daughters(ms[:1], None, 0.1, box=sy.box)
        bad = s["types"].copy()
        bad[0] = 3
        with pytest.raises(T.TTCFError):
            c.spawn_confined(ms[:1], bad, s["lattice"], sy.box, al[:1], 0.1)
        with pytest.raises(T.TTCFError):
            c.spawn_confined(ms[:1], np.zeros_like(s["types"]), s["lattice"], sy.box, al[:1], 0.1)
        with pytest.raises(T.TTCFError):
            c.spawn_confined(ms[:1], s["types"], s["lattice"], (5.0, sy.box[1], sy.box[2]), al[:1], 0.1)
        bid = c.spawn_confined(ms[:1], s["types"], s["lattice"], sy.box, al[:1], 0.1)
        with pytest.raises(T.TTCFError):
            c.run(5)            # confined daughters run in one call
        c.run()
        with pytest.raises(T.TTCFError):
            c.viscosity(bid)
        with pytest.raises(T.TTCFError):
            c.response_obs(bid, NOBS)


def test_equilibrium_friction_matches_the_oracle(ttcf, chan):
    """The equilibrium friction coefficient xi_0 (Eq. 12 by the equilibrium
    method): zero-shear daughters of the oracle mothers with one mapping are
    equilibrium trajectories; the device's slip/force correlations and the
    Maxwell fit equal the oracle's estimator applied to the same device
    series.  A sheared batch is refused."""
    T = ttcf
    s, sy, ms, al = chan
    n, se, lag = 400, 2, 60
    svals = np.linspace(0.2, 4.0, 12)
    with cctx(T, n_steps=n, sample_every=se, mapping_mask=1) as c:
        bid = c.spawn_confined(ms, s["types"], s["lattice"], sy.box, al, 0.0)
        c.run()
        Bg, _ = c.daughter_series(bid, ms.shape[0], NOBS)
        got = [c.friction_equilibrium(bid, w, lag, svals) for w in (0, 1)]
    ds = se * 0.005
    area = sy.box[0] * sy.box[2]
    for w in (0, 1):
        n_layer = len(oc.inner_layer(s["types"], s["lattice"], w))
        slabs = orr.adjacent_slabs(sy.box[1], H, w)
        ref = orr.friction_equilibrium(Bg, area, n_layer, slabs, w, ds, lag, svals)
        assert np.allclose(got[w]["c_dvf"], ref["c_dvf"], rtol=1e-9, atol=1e-12 * np.abs(ref["c_dvf"]).max())
        assert np.allclose(got[w]["c_dvdv"], ref["c_dvdv"], rtol=1e-9, atol=1e-12 * np.abs(ref["c_dvdv"]).max())
        assert np.allclose(got[w]["zeta_s"], ref["zeta_s"], rtol=1e-7)
        for k in ("xi0", "zeta0", "tau_m", "xi_ratio"):
            assert got[w][k] == pytest.approx(ref[k], rel=1e-6), k
        # velocity and force uncorrelated at equal times (time reversal), to noise
        assert abs(got[w]["c_dvf"][0]) < 0.2 * np.abs(got[w]["c_dvf"]).max()
    with cctx(T, n_steps=20, mapping_mask=1) as c:
        bid = c.spawn_confined(ms[:1], s["types"], s["lattice"], sy.box, al[:1], 0.05)
        c.run()
        with pytest.raises(T.TTCFError) as e:
            c.friction_equilibrium(bid, 0, 5, svals)
        assert e.value.status == T.TTCF_E_INVALID
