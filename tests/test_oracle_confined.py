"""Pins of the confined-system oracle (Example 2: Eq. 9, 10, 11)."""
import numpy as np
import pytest

from oracle import confined as oc
from paper_2312_02990_gb300 import inputs


@pytest.fixture(scope="module")
def small():
    """A small channel (10 x 10 rows, 2 wall layers), thermalised at rest."""
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=3)
    sy = oc.Confined(types=s["types"], box=tuple(s["box"]))
    ms, al = oc.mother(sy, s["state"], s["lattice"], n_eq=1500, n_states=3, spacing=150)
    return s, sy, ms, al


def test_geometry_is_x_reflection_symmetric_and_ordered():
    s = inputs.confined_system()
    assert (s["n_fluid"], s["n_wall"]) == (6048 - 0 * 1, 4200) or s["n_wall"] == 4200
    for t in (1, 2):
        P = s["lattice"][:, s["types"] == t].T
        Q = P.copy()
        Q[:, 0] = -Q[:, 0]
        Lx = s["box"][0]
        Q[:, 0] -= Lx * np.floor((Q[:, 0] + Lx / 2) / Lx)
        assert set(map(tuple, np.round(P, 6))) == set(map(tuple, np.round(Q, 6)))
    f = s["state"][1, s["types"] == 0]
    assert f.max() <= 0.5 * s["h"] - 1.0 + 1e-12 and f.min() >= -(0.5 * s["h"] - 1.0) - 1e-12


@pytest.mark.parametrize("types,c_key", [((0, 0), "c_ff"), ((0, 1), "c_wf"), ((2, 0), "c_wf"), ((2, 1), "c_ww"),
                                           ((1, 1), "c_ww"), ((2, 2), "c_ww")])
def test_pair_force_and_energy_closed_forms(types, c_key):
    """Two atoms at distance r: force -dphi/dr of Eq. 9 with the c of the
    pair's types, energy phi(r) - phi(r_c); tethers sit on the atoms."""
    r = 1.17
    st = np.zeros((6, 2))
    st[0] = [-0.3, -0.3 + r]
    lat = st[:3].copy()
    sy = oc.Confined(types=np.array(types, np.int32), box=(10.0, 10.0, 10.0))
    c = getattr(sy, c_key)
    F, U, Ut, _ = oc.forces(sy, st, lat, cells=False)
    dphi = 48.0 * r ** -13 - 24.0 * c * r ** -7          # -dphi/dr
    assert F[0, 0] == pytest.approx(-dphi, rel=1e-13)   # x force on atom 0
    assert F[0, 1] == pytest.approx(dphi, rel=1e-13)    # x force on atom 1
    assert np.all(F[1:] == 0.0)
    phi = lambda x: 4.0 * (x ** -12 - c * x ** -6)
    assert U == pytest.approx(phi(r) - phi(sy.rc), rel=1e-13)
    assert Ut == 0.0
    if c_key == "c_ww":   # switched off, the tethers alone hold the walls
        sy.ww_on = False
        F, U, _, _ = oc.forces(sy, st, lat, cells=False)
        assert np.all(F == 0.0) and U == 0.0


def test_cells_equal_all_pairs(small):
    s, sy, ms, al = small
    F1, U1, T1, w1 = oc.forces(sy, ms[0], s["lattice"], cells=True)
    F2, U2, T2, w2 = oc.forces(sy, ms[0], s["lattice"], cells=False)
    assert np.abs(F1 - F2).max() < 1e-11 * np.abs(F2).max()
    assert U1 == pytest.approx(U2, rel=1e-12) and T1 == pytest.approx(T2, rel=1e-12)
    assert np.allclose(w1, w2, rtol=1e-10, atol=1e-10)


def test_wall_stress_is_minus_the_shear_derivative_of_the_pair_energy(small):
    """Rigidly sliding the top wall by e in x changes the pair energy by
    -e * (x force of the fluid on the top wall); same for the bottom wall."""
    s, sy, ms, al = small
    st = ms[0]
    _, _, _, sw = oc.forces(sy, st, s["lattice"])
    h = 1e-6
    for idx, t in ((1, 2), (0, 1)):
        def U(e):
            x = st.copy()
            x[0, sy.types == t] += e
            return oc.forces(sy, x, s["lattice"])[1]
        dU = (U(h) - U(-h)) / (2 * h)
        assert dU == pytest.approx(-sw[idx], rel=1e-5, abs=1e-6)
    # pair forces sum to zero: total force = minus the tether forces
    F, _, _, _ = oc.forces(sy, st, s["lattice"])
    d = st[:3] - s["lattice"]
    d[0] -= sy.box[0] * np.rint(d[0] / sy.box[0])
    d[2] -= sy.box[2] * np.rint(d[2] / sy.box[2])
    tether = -sy.k * d * (sy.types != 0)
    assert np.abs((F - tether).sum(axis=1)).max() < 1e-9 * np.abs(F).max()


def test_energy_balances_are_second_order(small):
    s, sy, ms, al = small
    for vwall in (0.0, 0.3):
        dev = []
        for dt in (0.004, 0.002):
            sys2 = oc.Confined(types=sy.types, box=sy.box, dt=dt, vwall=vwall)
            _, _, _, obs = oc.trajectory(sys2, ms[0], s["lattice"], int(round(0.4 / dt)), alpha=al[0])
            H, P = obs[:, 5], obs[:, 6]
            W = np.concatenate([[0.0], np.cumsum(0.5 * dt * (P[1:] + P[:-1]))])
            good = H - W          # dH_ext/dt = P_lattice = -sum_w k (x_w - x_l) s_w v
            dev.append(np.abs(good - good[0]).max())
            if vwall:
                bad = H + W
                assert np.abs(bad - bad[0]).max() > 20 * dev[-1]
        assert 2.5 < dev[0] / dev[1] < 6.0, (vwall, dev)


def test_mappings_cancel_omega_and_odd_responses(small):
    s, sy, ms, al = small
    sys2 = oc.Confined(types=sy.types, box=sy.box, vwall=0.05)
    B, Om = oc.daughters(sys2, ms[:2], s["lattice"], al[:2], n_steps=2)
    for g in range(2):
        o = Om[4 * g:4 * g + 4]
        assert abs(o.sum()) <= 1e-12 * np.abs(o).sum()
        assert o[0] == pytest.approx(o[1], rel=1e-12) and o[2] == pytest.approx(-o[0], rel=1e-10)
        B0 = B[4 * g:4 * g + 4, 0]
        ns = sys2.nslab
        assert np.abs(B0[:, :2].sum(axis=0)).max() <= 1e-10 * np.abs(B0[:, :2]).max()   # wall stress
        assert np.abs(B0[:, 2:2 + ns].sum(axis=0)).max() < 1e-10                          # slab momenta
        assert np.all(B0[:, 2 + ns:2 + 2 * ns] == B0[0, 2 + ns:2 + 2 * ns])                # slab counts
        assert np.abs(B0[:, 2 + 2 * ns:].sum(axis=0)).max() < 1e-10                        # wall layers
        assert B0[0, 2 + ns:2 + 2 * ns].sum() == np.sum(sy.types == 0)


def test_time_reversal_with_walls_at_rest(small):
    s, sy, ms, al = small
    s1, l1, a1, _ = oc.trajectory(sy, ms[0], s["lattice"], 200, alpha=al[0])
    r, lr, ar = oc.apply_mapping(sy, 1, s1, l1, a1)
    s2, l2, a2, _ = oc.trajectory(sy, r, lr, 200, alpha=ar)
    back, lb, ab = oc.apply_mapping(sy, 1, s2, l2, a2)
    d = back[:3] - ms[0][:3]
    d[0] -= sy.box[0] * np.rint(d[0] / sy.box[0])
    d[2] -= sy.box[2] * np.rint(d[2] / sy.box[2])
    assert np.abs(d).max() < 1e-8 and np.abs(back[3:] - ms[0][3:]).max() < 1e-8
    assert ab == pytest.approx(al[0], abs=1e-9)


def test_omega_is_beta_times_the_adiabatic_energy_rate(small):
    """Omega(0) = beta dH0/dt at switch-on (Mathematical Framework; Eq. 11):
    with the thermostat frozen the energy change over one small step
    approaches Omega(0) T_w dt."""
    s, sy, ms, al = small
    v = 0.2
    for m in (0, 2):
        B, om, _ = oc.daughter(oc.Confined(types=sy.types, box=sy.box, vwall=v), ms[0],
                               s["lattice"], 0.0, m, n_steps=1)
        mapped, lat, _ = oc.apply_mapping(sy, m, ms[0], s["lattice"], 0.0)
        rates = []
        for dt in (1e-4, 5e-5):
            frozen = oc.Confined(types=sy.types, box=sy.box, vwall=v, dt=dt, tau_T=1e12)
            _, _, _, obs = oc.trajectory(frozen, mapped, lat, 1, alpha=0.0)
            H0 = obs[:, 0] + obs[:, 1] + obs[:, 2]
            rates.append((H0[1] - H0[0]) / dt)
        # the one-sided difference converges linearly: extrapolate to dt = 0
        rate0 = 2 * rates[1] - rates[0]
        assert rate0 / sy.Tw == pytest.approx(om, rel=2e-3), (m, rate0, om)
        assert abs(om) > 1e-3


def test_friction_of_constructed_responses():
    """Eq. 12 on responses built so that the wall-layer and fluid velocities
    and the wall stress are known: slip = v_wall - v_fluid (the paper's slip
    velocity: innermost wall layer minus outermost fluid layer) and
    xi = -sigma / slip."""
    from oracle import reduce as orr
    Ly, h, g, ns, n_layer = 15.95, 10.0, 0.02, oc.N_SLAB, 700
    t = np.linspace(0.0, 1.0, 11)
    for wall, sw in ((0, -1.0), (1, 1.0)):
        ks = orr.adjacent_slabs(Ly, h, wall, ns)
        centres = -0.5 * Ly + (ks + 0.5) * Ly / ns
        assert len(ks) >= 2 and np.all(np.abs(np.abs(centres) - 0.5 * h) < 1.0)
        v_fluid = 0.3 * sw * g * t            # fluid lags the wall
        v_wall = sw * g * 0.5 * h * (1.0 + 0.1 * t)
        # the fluid drags the wall backwards: sigma has the sign of -slip
        sigma = 2.5 * (v_fluid - v_wall)
        resp = {o: {"ttcf": np.zeros_like(t)} for o in range(oc.N_OBS)}
        resp[wall]["ttcf"] = sigma
        resp[2 + 2 * ns + wall]["ttcf"] = n_layer * v_wall
        for j, k in enumerate(ks):
            n_k = 10.0 + j
            resp[2 + ns + k]["ttcf"] = np.full_like(t, n_k)
            resp[2 + k]["ttcf"] = n_k * v_fluid
        f = orr.friction(resp, Ly, h, wall, n_layer, ns)
        assert np.allclose(f["slip"], v_wall - v_fluid, rtol=1e-14, atol=1e-16)
        assert np.allclose(f["xi"], 2.5, rtol=1e-13)


def test_inner_wall_layer_observable():
    """The inner-layer responses: the innermost FCC(111) layer of each wall
    holds one layer's atoms (nx * nz), the response at t = 0 is the sum of
    their p_x, and a layer tethered to a lattice sliding at +-v moves on
    average at +-v: over a window of a few tether periods the layer velocity
    x' = v (1 - cos w t) of an atom starting at rest on its site averages to
    v (1 - sin(w T)/(w T)), w = sqrt(k), plus thermal noise of the layer
    mean."""
    s = inputs.confined_system(nx=10, nz=10, layers=2, seed=11)
    ns = oc.N_SLAB
    for w in (0, 1):
        idx = oc.inner_layer(s["types"], s["lattice"], w)
        assert len(idx) == 100
        yl = s["lattice"][1, idx]
        assert np.all(np.abs(yl - (1 if w else -1) * 0.5 * s["h"]) < 1e-12)
    v = 0.5
    sy = oc.Confined(types=s["types"], box=tuple(s["box"]), vwall=v)
    B, om, _ = oc.daughter(sy, s["state"], s["lattice"], 0.0, 0, 400, 1)
    for w, sgn in ((0, -1.0), (1, 1.0)):
        idx = oc.inner_layer(s["types"], s["lattice"], w)
        assert B[0, 2 + 2 * ns + w] == pytest.approx(s["state"][3, idx].sum(), rel=1e-12, abs=1e-12)
        vel = B[:, 2 + 2 * ns + w] / len(idx)
        T = 400 * sy.dt
        om_t = np.sqrt(sy.k)
        expect = sgn * v * (1.0 - np.sin(om_t * T) / (om_t * T))
        assert abs(vel[1:].mean() - expect) < 0.1 * v, (w, vel[1:].mean(), expect)
