"""Pins of the FP64 oracle's planar elongational flow against facts fixed by
mechanics, independent of its own formulas: a closed-form lattice sum for an
affinely deformed crystal, the extended-energy balance of Eq. 5 with
grad u = diag(eps, 0, -eps), the reduction to the zero-field dynamics, the
x <-> z exchange symmetry of the flow, and the mapping set's cancellation of
Omega(0)."""
import numpy as np
import pytest

import oracle
from elong_lattice import fcc_vectors, lattice_sums
from paper_2312_02990_gb300 import inputs

RC = 2.0 ** (1.0 / 6.0)
XZ = 16                       # mapping code of the x <-> z exchange
ELONG_SET = (0, 1, 16, 17)    # identity, p -> -p, exchange, both


def bulk(N, **kw):
    return oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)), **kw)


def _eq_state(N=256, seed=7, n_eq=3000):
    b = bulk(N)
    ms, al = oracle.mother(b, inputs.initial_state(N, seed), n_eq, 1, 10)
    return b, ms[0], al[0]


def test_affine_lattice_follows_the_closed_form():
    """A perfect FCC crystal at rest stays a perfect (deformed) crystal: every
    site is an inversion centre, so all forces vanish, momenta stay zero,
    positions follow r(t) = diag(e^{eps t}, 1, e^{-eps t}) r(0), alpha falls
    at the constant rate -gT/Q, and P_xx - P_zz and U are lattice sums over
    the deformed neighbour shell (which the compression brings inside r_c)."""
    N, eps, n = 256, 0.5, 300
    b = bulk(N)
    L = b.L[0]
    st = np.zeros((6, N))
    st[:3] = inputs.fcc_lattice(N)
    fin, a_end, obs = oracle.trajectory_elong(b, st, n, eps, alpha=0.0)
    a = L / inputs.fcc_cells_for(N)
    R0 = fcc_vectors(a, 2.0 * RC)
    h = b.dt
    interacting = 0
    for k in range(0, n + 1, 25):
        B, U = lattice_sums(R0, N, b.V, k * h, eps)
        interacting += U > 0
        assert obs[k, 4] == pytest.approx(B, rel=1e-10, abs=1e-12)
        assert obs[k, 1] == pytest.approx(U, rel=1e-10, abs=1e-12)
        assert obs[k, 2] == pytest.approx(-b.dof * b.T * k * h / b.Q, rel=1e-12)
        assert obs[k, 6] == pytest.approx(L * np.exp(eps * k * h), rel=1e-14)
        assert obs[k, 7] == pytest.approx(L * np.exp(-eps * k * h), rel=1e-14)
    assert interacting >= 4   # the closed form is not trivially zero
    assert np.abs(fin[3:]).max() < 1e-12
    E = np.array([np.exp(eps * n * h), 1.0, np.exp(-eps * n * h)])[:, None]
    Lt = np.array([obs[n, 6], L, obs[n, 7]])[:, None]
    d = fin[:3] - E * st[:3]
    d -= Lt * np.rint(d / Lt)
    assert np.abs(d).max() < 1e-10


def test_elongational_energy_balance_pins_the_sign_of_the_work():
    """dH_ext/dt = -V grad u : P = -eps V (P_xx - P_zz) for the Eq. 5 SLLOD
    flow with Nose-Hoover; the residual is second order in dt, and with the
    opposite sign the balance fails by orders of magnitude."""
    b, st, a0 = _eq_state()
    eps = 0.5
    dev = []
    for dt in (0.0025, 0.00125):
        bb = oracle.Bulk(n=b.n, L=b.L, dt=dt)
        _, _, obs = oracle.trajectory_elong(bb, st, int(round(1.0 / dt)), eps, alpha=a0)
        H, P = obs[:, 8], obs[:, 4]
        I = np.concatenate([[0.0], np.cumsum(0.5 * dt * (P[1:] + P[:-1]))])
        good = H + eps * bb.V * I
        bad = H - eps * bb.V * I
        dev.append(np.abs(good - good[0]).max())
        assert np.abs(bad - bad[0]).max() > 100 * dev[-1]
    assert 2.5 < dev[0] / dev[1] < 6.0


def test_zero_rate_is_the_zero_field_dynamics():
    """At eps = 0 the elongational step is the zero-shear step of Eq. 5."""
    b, st, a0 = _eq_state()
    s1, a1, _, o1 = oracle.trajectory(b, st, 200, gamma=0.0, alpha=a0)
    s2, a2, o2 = oracle.trajectory_elong(b, st, 200, 0.0, alpha=a0)
    assert np.abs(s1 - s2).max() < 1e-12
    assert a1 == pytest.approx(a2, abs=1e-14)
    assert np.abs(o1[:, 0] - o2[:, 0]).max() < 1e-10   # sum p^2


def test_exchange_maps_the_flow_onto_the_opposite_rate():
    """Exchanging x and z turns diag(eps, 0, -eps) into diag(-eps, 0, eps):
    the trajectory of the exchanged state at -eps is the exchanged trajectory
    at +eps, and P_xx - P_zz changes sign along it."""
    b, st, a0 = _eq_state()
    eps = 0.2
    s1, a1, o1 = oracle.trajectory_elong(b, st, 150, eps, alpha=a0)
    xs, xa = oracle.apply_mapping(b, XZ, st, a0)
    s2, a2, o2 = oracle.trajectory_elong(b, xs, 150, -eps, alpha=xa)
    back = s2[[2, 1, 0, 5, 4, 3]]
    assert np.abs(back - s1).max() < 1e-9
    assert a2 == pytest.approx(a1, abs=1e-10)
    assert np.abs(o2[:, 4] + o1[:, 4]).max() < 1e-9
    assert np.abs(o2[:, 6] - o1[:, 7]).max() < 1e-12   # Lx at -eps = Lz at +eps


def test_box_keeps_its_volume_and_its_atoms_and_momentum():
    b, st, a0 = _eq_state()
    eps = -0.3                # compression along x, stretching along z
    n = 400
    fin, _, obs = oracle.trajectory_elong(b, st, n, eps, alpha=a0)
    L = b.L[0]
    assert np.allclose(obs[:, 6] * obs[:, 7], L * L, rtol=1e-14, atol=0)
    Lt = np.array([obs[n, 6], L, obs[n, 7]])[:, None]
    assert np.all(fin[:3] >= -0.5 * Lt) and np.all(fin[:3] < 0.5 * Lt)
    assert np.abs(st[3:].sum(axis=1)).max() < 1e-10
    assert np.abs(fin[3:].sum(axis=1)).max() < 1e-9


def test_elongational_mappings_cancel_omega():
    """Omega(0) = -eps V (P_xx - P_zz)/T: time reversal keeps P_xx - P_zz,
    the x <-> z exchange negates it, so the four daughters of a group sum
    to zero, and B(0) is the pressure difference of the mapped state."""
    b = bulk(256)
    eps = 1e-3
    for st in inputs.jittered_states(256, 3, seed=31, amp=0.1):
        om, b0 = [], []
        for m in ELONG_SET:
            B, o, _, _ = oracle.daughter_elong(b, st, 0.1, m, eps, 3)
            P = oracle.pressure(b, oracle.apply_mapping(b, m, st)[0])[0]
            assert B[0] == pytest.approx(P[0] - P[2], rel=1e-12)
            assert o == pytest.approx(-eps * b.V * (P[0] - P[2]) / b.T, rel=1e-12)
            om.append(o)
            b0.append(B[0])
        assert om[1] == pytest.approx(om[0], rel=1e-12)
        assert om[2] == pytest.approx(-om[0], rel=1e-10)
        assert abs(sum(om)) <= 1e-10 * sum(abs(o) for o in om)
        assert abs(sum(b0)) <= 1e-10 * sum(abs(v) for v in b0)


def test_ensemble_driver_matches_single_daughters():
    b, st, a0 = _eq_state()
    ms = np.stack([st, st])
    B, Om = oracle.daughters_elong(b, ms, [a0, a0], [0.05, -0.05], 20, sample_every=5)
    assert B.shape == (8, 5) and Om.shape == (8,)
    for d in range(8):
        g, m = divmod(d, 4)
        Bd, od, _, _ = oracle.daughter_elong(b, ms[g], a0, ELONG_SET[m], [0.05, -0.05][g], 20,
                                             sample_every=5)
        assert np.array_equal(B[d], Bd) and Om[d] == od


def test_elongational_ttcf_reduces_to_green_kubo_at_weak_field(eq_mothers_256):
    """At eps -> 0, Eq. 1 with Omega(0) = -eps V B(0)/T and the mapped set's
    <B(0)> = 0 gives eta_1(t) = (V / 4T) int_0^t <B(0) B(s)> ds, the
    Green-Kubo integral of B = P_xx - P_zz along the zero-field trajectories
    of the same mapped states (a wrong sign or factor of Omega, or of the
    1/(4 eps) of eta_1, fails it)."""
    b, ms, al = eq_mothers_256
    n, eps = 120, 1e-8
    B, Om = oracle.daughters_elong(b, ms[:16], al[:16], eps, n)
    eta1 = -oracle.responses(B, Om, 4, b.dt)["ttcf"] / (4.0 * eps)
    B0, _ = oracle.daughters_elong(b, ms[:16], al[:16], 0.0, n)
    acf = (B0[:, :1] * B0).mean(axis=0)
    gk = b.V / (4.0 * b.T) * np.concatenate([[0.0], np.cumsum(0.5 * b.dt * (acf[1:] + acf[:-1]))])
    assert np.abs(gk).max() > 0.1
    assert np.allclose(eta1[1:], gk[1:], rtol=1e-5, atol=1e-7 * np.abs(gk).max())
