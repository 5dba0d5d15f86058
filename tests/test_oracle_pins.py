"""Pins of the FP64 oracle against facts fixed by the paper and by mechanics,
independent of the oracle's own formulas (closed forms, energy derivatives,
conservation laws, exact symmetries, brute force, Green-Kubo)."""
import numpy as np
import pytest

import oracle
from paper_2312_02990_gb300 import inputs

RC = 2.0 ** (1.0 / 6.0)


def bulk(N, **kw):
    return oracle.Bulk(n=N, L=tuple(inputs.bulk_box(N)), **kw)


# ---------------------------------------------------------------- Eq. 6 ----
def test_wca_closed_forms():
    # phi(sigma) = eps (the shift is +eps), F(sigma) = 24 eps/sigma.
    phi1, f1 = oracle.wca(1.0)
    assert phi1 == pytest.approx(1.0, abs=1e-15)
    assert f1 * 1.0 == pytest.approx(24.0, abs=1e-13)
    # Continuity at r_c: phi -> 0 and F -> 0 from below; zero beyond.
    phic, fc = oracle.wca(RC * RC * (1 - 1e-12))
    assert abs(phic) < 1e-10 and abs(fc) < 1e-9
    assert oracle.wca(RC * RC * 1.0001) == (0.0, 0.0)
    # Minimum of the LJ part sits at r_c: phi(r_c) - 1 = -eps.
    # F = -dphi/dr by central differences at several r.
    for r in (0.9, 0.97, 1.05, 1.1):
        h = 1e-6
        dphi = (oracle.wca((r + h) ** 2)[0] - oracle.wca((r - h) ** 2)[0]) / (2 * h)
        assert oracle.wca(r * r)[1] * r == pytest.approx(-dphi, rel=1e-7)


# ------------------------------------------------ forces, images, virial ----
@pytest.mark.parametrize("N", [108, 256])
def test_cells_equal_brute_force_with_le_offsets(N):
    b = bulk(N)
    st = inputs.jittered_states(N, 3, seed=11, amp=0.12)
    rng = np.random.default_rng(5)
    for k in range(3):
        delta = rng.uniform(-0.5, 0.5) * b.L[0]
        Fc, Wc, Uc = oracle.forces(b, st[k], delta, brute=False)
        Fb, Wb, Ub = oracle.forces(b, st[k], delta, brute=True)
        assert np.abs(Fc - Fb).max() <= 1e-12 * np.abs(Fb).max()
        assert np.allclose(Wc, Wb, rtol=1e-12, atol=1e-12)
        assert Uc == pytest.approx(Ub, rel=1e-12)
        assert Uc > 0  # jitter of 0.12 creates overlaps


def test_two_atoms_across_the_le_boundary():
    """Atom j sits near the bottom face; its image above is shifted by +delta
    in x.  The only interacting image is at (x_j + delta, y_j + Ly)."""
    b = bulk(256)
    L = b.L[0]
    delta = 0.3 * L
    # a 2-atom system in the box of the N=256 state point
    b2 = oracle.Bulk(n=2, L=b.L, use_cells=False)
    s = np.zeros((6, 2))
    xi, yi = 0.1, 0.5 * L - 0.1
    xj, yj = xi - delta + 0.5, -0.5 * L + 0.3
    s[0] = [xi, xj]; s[1] = [yi, yj]; s[2] = [0.0, 0.05]
    F, W, U = oracle.forces(b2, s, delta)
    d = np.array([xi - (xj + delta), yi - (yj + L), 0.0 - 0.05])  # (-0.5, -0.4, -0.05)
    r2 = d @ d
    phi, for_ = oracle.wca(r2)
    assert r2 < RC * RC
    assert np.allclose(F[:, 0], for_ * d, rtol=1e-13)
    assert np.allclose(F[:, 1], -for_ * d, rtol=1e-13)
    assert U == pytest.approx(phi, rel=1e-14)
    assert W[3] == pytest.approx(for_ * d[0] * d[1], rel=1e-13)
    # with delta = 0 the same pair is out of range
    F0, _, U0 = oracle.forces(b2, s, 0.0)
    assert U0 == 0.0


def test_newton_third_law_and_cluster_virial():
    b = bulk(256)
    st = inputs.jittered_states(256, 1, seed=3, amp=0.12)[0]
    F, W, U = oracle.forces(b, st, 0.37 * b.L[0])
    assert np.abs(F.sum(axis=1)).max() < 1e-10 * np.abs(F).max()
    # Isolated cluster in a big box: W_ab = sum_i r_i,a F_i,b exactly.
    rng = np.random.default_rng(2)
    n = 40
    pos = rng.uniform(-1.6, 1.6, size=(3, n))
    big = oracle.Bulk(n=n, L=(50.0, 50.0, 50.0), use_cells=False)
    s = np.zeros((6, n)); s[:3] = pos
    Fc, Wc, _ = oracle.forces(big, s)
    idx = {0: (0, 0), 1: (1, 1), 2: (2, 2), 3: (0, 1), 4: (0, 2), 5: (1, 2)}
    for k, (a, c) in idx.items():
        assert Wc[k] == pytest.approx(np.sum(pos[a] * Fc[c]), rel=1e-10, abs=1e-9)


def test_virial_is_minus_strain_derivative_of_energy():
    """Shear strain eps: x -> x + eps*y with Lees-Edwards offset eps*Ly gives
    dU/deps = -W_xy; isotropic scaling gives dU/dlambda = -(Wxx+Wyy+Wzz).
    This pins the virial's sign, its 1/2 and the LE image convention."""
    N = 256
    b = bulk(N)
    st = inputs.jittered_states(N, 1, seed=8, amp=0.12)[0]
    _, W, _ = oracle.forces(b, st, 0.0)

    def U_shear(e):
        s = st.copy()
        s[0] = s[0] + e * s[1]
        return oracle.forces(b, s, e * b.L[1])[2]

    h = 1e-6
    dU = (U_shear(h) - U_shear(-h)) / (2 * h)
    assert dU == pytest.approx(-W[3], rel=1e-6)

    def U_scale(lam):
        bl = oracle.Bulk(n=N, L=tuple(np.asarray(b.L) * lam))
        s = st.copy(); s[:3] *= lam
        return oracle.forces(bl, s, 0.0)[2]

    dUl = (U_scale(1 + h) - U_scale(1 - h)) / (2 * h)
    assert dUl == pytest.approx(-(W[0] + W[1] + W[2]), rel=1e-6)


# ----------------------------------------------------------- integrator ----
def _eq_state(N=256, seed=7, n_eq=3000):
    b = bulk(N)
    ms, al = oracle.mother(b, inputs.initial_state(N, seed), n_eq, 1, 10)
    return b, ms[0], al[0]


def test_nve_energy_error_is_second_order():
    b, st, _ = _eq_state()
    dev = []
    for dt in (0.0025, 0.00125):
        bb = oracle.Bulk(n=b.n, L=b.L, dt=dt, tau_T=1e12)
        _, _, _, obs = oracle.trajectory(bb, st, int(round(1.0 / dt)), alpha=0.0)
        E = 0.5 * obs[:, 0] + obs[:, 1]
        dev.append(np.abs(E - E[0]).max())
        assert abs(E[-1] - E[0]) < 5e-4 * b.n  # no drift beyond the fluctuation
    assert 2.8 < dev[0] / dev[1] < 5.5


def test_nvt_extended_energy_is_conserved():
    b, st, a0 = _eq_state()
    dev = []
    for dt in (0.0025, 0.00125):
        bb = oracle.Bulk(n=b.n, L=b.L, dt=dt)
        _, _, _, obs = oracle.trajectory(bb, st, int(round(1.0 / dt)), alpha=a0)
        dev.append(np.abs(obs[:, 7] - obs[0, 7]).max())
    assert dev[0] < 0.05 and 2.5 < dev[0] / dev[1] < 6.0


def test_sheared_energy_balance_pins_the_sign_of_pxy():
    """dH_ext/dt = -gamma V P_xy for SLLOD + Nose-Hoover (Eq. 5); with the
    opposite sign the balance fails by orders of magnitude."""
    b, st, a0 = _eq_state()
    g = 0.5
    dev = []
    for dt in (0.0025, 0.00125):
        bb = oracle.Bulk(n=b.n, L=b.L, dt=dt)
        _, _, _, obs = oracle.trajectory(bb, st, int(round(1.0 / dt)), gamma=g, alpha=a0)
        H, P = obs[:, 7], obs[:, 4]
        I = np.concatenate([[0.0], np.cumsum(0.5 * dt * (P[1:] + P[:-1]))])
        good = H + g * bb.V * I
        bad = H - g * bb.V * I
        dev.append(np.abs(good - good[0]).max())
        assert np.abs(bad - bad[0]).max() > 100 * dev[-1]
    assert 2.5 < dev[0] / dev[1] < 6.0


def test_time_reversal_at_zero_field():
    """Mapping 1 (p -> -p, alpha -> -alpha) reverses the zero-field dynamics:
    n steps forward, map, n steps, map back = the start (Eq. 3, 5)."""
    b, st, a0 = _eq_state()
    s1, a1, _, _ = oracle.trajectory(b, st, 300, alpha=a0)
    r, ar = oracle.apply_mapping(b, 1, s1, a1)
    s2, a2, _, _ = oracle.trajectory(b, r, 300, alpha=ar)
    back, ab = oracle.apply_mapping(b, 1, s2, a2)
    d = back[:3] - st[:3]
    d -= np.asarray(b.L)[:, None] * np.rint(d / np.asarray(b.L)[:, None])
    assert np.abs(d).max() < 1e-9
    assert np.abs(back[3:] - st[3:]).max() < 1e-9
    assert ab == pytest.approx(a0, abs=1e-9)


def test_total_momentum_stays_zero_under_shear():
    b, st, a0 = _eq_state()
    s1, _, _, _ = oracle.trajectory(b, st, 400, gamma=0.3, alpha=a0)
    assert np.abs(st[3:].sum(axis=1)).max() < 1e-10
    assert np.abs(s1[3:].sum(axis=1)).max() < 1e-9


# -------------------------------------------------------------- Eq. 3 ----
def test_mappings_cancel_omega_and_pxy_exactly():
    b = bulk(256)
    st = inputs.jittered_states(256, 4, seed=21, amp=0.1)
    for k in range(4):
        P = [oracle.pressure(b, oracle.apply_mapping(b, m, st[k])[0])[0][3] for m in range(4)]
        kin = [np.sum(oracle.apply_mapping(b, m, st[k])[0][3] *
                      oracle.apply_mapping(b, m, st[k])[0][4]) for m in range(4)]
        # kinetic parts negate bitwise, configurational parts up to summation order
        assert kin[0] == kin[1] == -kin[2] == -kin[3]
        assert abs(sum(P)) <= 1e-12 * sum(abs(p) for p in P)
        assert P[0] == pytest.approx(P[1], rel=1e-14)
        assert P[2] == pytest.approx(-P[0], rel=1e-10)
    # m3 = m1 o m2, and alpha flips for the time-reversing mappings only
    s = st[0]
    a = 0.123
    m2, a2 = oracle.apply_mapping(b, 2, s, a)
    m12, a12 = oracle.apply_mapping(b, 1, m2, a2)
    m3, a3 = oracle.apply_mapping(b, 3, s, a)
    assert np.array_equal(m12, m3) and a12 == a3 == -a and a2 == a
    assert oracle.apply_mapping(b, 3, s, a, reset_alpha=True)[1] == 0.0


def test_daughter_omega_definition():
    b = bulk(256)
    st = inputs.jittered_states(256, 1, seed=4, amp=0.1)[0]
    g = 1e-3
    B, om, _, _ = oracle.daughter(b, st, 0.0, 0, g, 5)
    P = oracle.pressure(b, st)[0][3]
    assert B[0] == pytest.approx(P, rel=1e-14)
    assert om == pytest.approx(-g * b.V * P / b.T, rel=1e-14)


# -------------------------------------------------------- Eq. 1, 2, 4 ----
def test_reduce_closed_forms():
    # Two groups of four; B linear in t -> trapezoid is exact.
    S, ds = 11, 0.1
    t = np.arange(S) * ds
    Om = np.array([1.0, 1.0, -1.0, -1.0, 2.0, 2.0, -2.0, -2.0])
    B = np.stack([(1 + k) * t for k in range(8)])
    r = oracle.responses(B, Om, 4, ds)
    corr = (Om[:, None] * B).mean(axis=0)
    assert np.allclose(r["corr"], corr)
    slope = np.mean(Om * (1 + np.arange(8)))
    assert np.allclose(r["ttcf"], slope * t ** 2 / 2, atol=1e-14)
    assert np.allclose(r["dav"], 4.5 * t)
    assert r["omega_mean"] == 0.0
    # Eq. 4 correction with nonzero <Omega>: subtracts <Omega><B(s)>.
    Om2 = Om + 0.5
    r2 = oracle.responses(B, Om2, 4, ds, corrected=True)
    expect = np.mean(Om2 * (1 + np.arange(8))) * t ** 2 / 2 - 0.5 * 4.5 * t ** 2 / 2
    assert np.allclose(r2["ttcf"], expect, atol=1e-13)


def test_standard_errors_of_a_textbook_sample():
    """The group standard error against a worked textbook example: the eight
    values 2, 4, 4, 4, 5, 5, 7, 9 have mean 5, population standard deviation
    2 and sample variance 32/7, so the standard error of their mean is
    sqrt(32/7)/sqrt(8) = sqrt(4/7).  Eight mother groups take these values
    as group means a_g of B; four mapped daughters per group add deviations
    c_m(s) = w_m (1 + 0.3 s) that cancel within the group, w = (1, 1, -1, -1),
    and Omega_{g,m} = a_g w_m, so each group's integrand is
    Y_g(s) = a_g (1/4) sum_m w_m c_m(s) = a_g (1 + 0.3 s), hence
        dav_se  = sqrt(4/7)                        (spread of D_g = a_g)
        corr_se = sqrt(4/7) (1 + 0.3 s)            (spread of Y_g)
        ttcf_se = sqrt(4/7) (1 + s ds + 0.15 s^2 ds)   (spread of J_g)
    A standard error taken over daughters, with ddof = 0 or over 4G instead of
    G samples gives another number."""
    a = np.array([2.0, 4, 4, 4, 5, 5, 7, 9])
    w = np.array([1.0, 1.0, -1.0, -1.0])
    S, ds = 9, 0.25
    s = np.arange(S)
    G = a.size
    B = np.zeros((4 * G, S))
    Om = np.zeros(4 * G)
    for g in range(G):
        for m in range(4):
            B[4 * g + m] = a[g] + w[m] * (1.0 + 0.3 * s)
            Om[4 * g + m] = a[g] * w[m]
    r = oracle.responses(B, Om, 4, ds)
    se = np.sqrt(4.0 / 7.0)
    assert np.allclose(r["dav"], 5.0, rtol=0, atol=1e-14)
    assert np.allclose(r["dav_se"], se, rtol=1e-14, atol=0)
    lin = 1.0 + 0.3 * s
    assert np.allclose(r["corr"], 5.0 * lin, rtol=1e-14)
    assert np.allclose(r["corr_se"], se * lin, rtol=1e-14)
    # J_g(s) = a_g + a_g int_0^t (1 + 0.3 s') = a_g (1 + t + 0.15 t^2 / ds), t = s ds
    # (the trapezoid rule is exact on a linear integrand)
    J = 1.0 + s * ds + 0.15 * s * s * ds
    assert np.allclose(r["ttcf"], 5.0 * J, rtol=1e-14)
    assert np.allclose(r["ttcf_se"], se * J, rtol=1e-13)
    # the paper's figure convention (over daughters) differs from the group SE
    assert not np.allclose(r["dav_se_daughters"], se)


def test_autocorrelation_closed_forms():
    """The equilibrium correlation (over trajectories and time origins)
    against series whose correlations are known exactly:
      alternating +-1:  <B(t)B(t+k)> = (-1)^k, B^2 = 1 so acf2 = 0, and the
                        trapezoid integral of (-1)^k vanishes at every lag;
      ramp B(t) = t, n samples:  with m = n - k origins,
                        <t (t+k)> = (m-1)(2m-1)/6 + k (m-1)/2;
      constant c:       acf = c^2 and the Green-Kubo integral is
                        (V/T) c^2 k ds."""
    n, lag = 50, 7
    alt = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    acf, acf2 = oracle.autocorrelation(np.stack([alt, -alt]), lag)
    assert np.array_equal(acf, (-1.0) ** np.arange(lag + 1))
    assert np.all(acf2 == 0.0)
    assert np.allclose(oracle.green_kubo(acf, 2.0, 0.5, 0.1), 0.0, atol=1e-15)
    ramp = np.arange(n, dtype=float)
    acf, _ = oracle.autocorrelation(ramp[None], lag)
    m = n - np.arange(lag + 1)
    k = np.arange(lag + 1)
    assert np.allclose(acf, (m - 1) * (2 * m - 1) / 6.0 + k * (m - 1) / 2.0, rtol=1e-14)
    acf, acf2 = oracle.autocorrelation(np.full((3, n), 1.5), lag)
    assert np.allclose(acf, 2.25) and np.allclose(acf2, 0.0)
    assert np.allclose(oracle.green_kubo(acf, 3.0, 0.75, 0.01), 3.0 / 0.75 * 2.25 * k * 0.01, rtol=1e-14)


def test_dav_standard_error_is_zero_at_t0(eq_mothers_256):
    b, ms, al = eq_mothers_256
    B, Om = oracle.daughters(b, ms[:8], al[:8], 1e-3, 40)
    r = oracle.responses(B, Om, 4, b.dt)
    assert abs(r["dav"][0]) < 1e-16 and r["dav_se"][0] < 1e-16
    assert abs(Om.sum()) <= 1e-12 * np.abs(Om).sum()
    # grows from zero during the transient (Fig. 8)
    assert 0 < r["dav_se"][10] < r["dav_se"][20] < r["dav_se"][40]


def test_ttcf_reduces_to_green_kubo_at_weak_field(eq_mothers_256):
    """Eq. 1 with Eq. 7 at gamma -> 0 is the Green-Kubo integral of Eq. 8
    evaluated on zero-field trajectories from the same mapped states."""
    b, ms, al = eq_mothers_256
    n = 120
    g = 1e-8
    B, Om = oracle.daughters(b, ms[:16], al[:16], g, n)
    eta = oracle.viscosity(oracle.responses(B, Om, 4, b.dt), g)["eta_ttcf"]
    B0, _ = oracle.daughters(b, ms[:16], al[:16], 0.0, n)
    acf = (B0[:, :1] * B0).mean(axis=0)
    gk = b.V / b.T * np.concatenate([[0.0], np.cumsum(0.5 * b.dt * (acf[1:] + acf[:-1]))])
    assert np.allclose(eta[1:], gk[1:], rtol=1e-5, atol=1e-7 * np.abs(gk).max())


def test_standard_errors_scale_with_the_field_as_in_eq_13_to_16(eq_mothers_256):
    """In the linear regime the integrand's spread grows in proportion to the
    field (Eq. 13: sigma(Omega(0) P_xy) = k1 gamma sqrt(...)), so the standard
    error of <Omega(0)B(s)> scales with gamma while that of the TTCF
    viscosity does not (Eq. 15-16).  (The direct average's spread is
    field-independent only in the steady state, not in this transient.)"""
    b, ms, al = eq_mothers_256
    n = 160
    r = {}
    for g in (1e-3, 1e-4):
        B, Om = oracle.daughters(b, ms[:24], al[:24], g, n)
        r[g] = oracle.responses(B, Om, 4, b.dt)
    s = slice(20, None)
    ratio = r[1e-3]["corr_se"][s] / r[1e-4]["corr_se"][s]
    assert np.all(np.abs(ratio / 10.0 - 1.0) < 0.02), ratio.min()
    eta_se = {g: r[g]["ttcf_se"][s] / g for g in r}
    assert np.all(np.abs(eta_se[1e-3] / eta_se[1e-4] - 1.0) < 0.02)


def test_ttcf_agrees_with_direct_average_at_high_shear(eq_mothers_256):
    """At strong field the direct average is precise and TTCF must agree
    with it (Example 1, Fig. 3; Example 2 at gamma = 1e-1)."""
    b, ms, al = eq_mothers_256
    g, n = 1.0, 200
    B, Om = oracle.daughters(b, ms, al, g, n)
    G = ms.shape[0]
    Bg = B.reshape(G, 4, -1)
    Og = Om.reshape(G, 4)
    Y = np.einsum("gm,gms->gs", Og, Bg) / 4
    J = Bg.mean(axis=1)[:, :1] + np.concatenate(
        [np.zeros((G, 1)), np.cumsum(0.5 * b.dt * (Y[:, 1:] + Y[:, :-1]), axis=1)], axis=1)
    Dg = Bg.mean(axis=1)
    for s in (100, 200):
        diff = J[:, s] - Dg[:, s]
        se = diff.std(ddof=1) / np.sqrt(G)
        assert abs(diff.mean()) < 2.0 * se, (s, diff.mean(), se)
    r = oracle.responses(B, Om, 4, b.dt)
    assert r["dav"][-1] < -5 * r["dav_se"][-1]  # a real, negative P_xy response


def test_mapping_keeps_positions_in_the_half_open_box():
    """x -> -x sends an atom on the face x = -L/2 to +L/2, which is the same
    periodic point; the mapped state stays in [-L/2, L/2)."""
    b = bulk(256)
    st = inputs.initial_state(256, 3)
    st[0, 0] = -0.5 * b.L[0]
    for m in (2, 3):
        out, _ = oracle.apply_mapping(b, m, st)
        assert out[0, 0] == -0.5 * b.L[0]
        assert np.all(out[0] >= -0.5 * b.L[0]) and np.all(out[0] < 0.5 * b.L[0])


# ------------------------------------------ mappings beyond Eq. 3 ----------
def _pressure_tensor(b, s):
    P, U, K2 = oracle.pressure(b, s)
    # components xx yy zz xy xz yz
    return P, U, K2


@pytest.mark.parametrize("m", range(32))
def test_every_mapping_is_an_isometry_with_the_tensor_law(m):
    """Each mapping code (exchange x <-> z, then reflections, then time
    reversal) keeps the kinetic and potential energy (an isometry of the
    cubic periodic box) and transforms the pressure tensor as a tensor:
    P'_xy = s_x s_y P_xy, or s_x s_y P_zy when x and z are exchanged, with
    s_a = -1 for a reflected axis; time reversal leaves P unchanged and
    negates alpha."""
    N = 256
    b = bulk(N)
    st = inputs.jittered_states(N, 1, seed=40 + m, amp=0.1)[0]
    st[3:] = np.random.default_rng(m).standard_normal((3, N))
    P, U, K2 = _pressure_tensor(b, st)
    out, a = oracle.apply_mapping(b, m, st, alpha=0.3)
    P2, U2, K22 = _pressure_tensor(b, out)
    assert U2 == pytest.approx(U, rel=1e-12)
    assert K22 == pytest.approx(K2, rel=1e-14)
    sx = -1.0 if m & 2 else 1.0
    sy = -1.0 if m & 4 else 1.0
    base = P[5] if m & 16 else P[3]      # P_zy = P_yz after the exchange
    assert P2[3] == pytest.approx(sx * sy * base, rel=1e-11, abs=1e-13)
    assert a == (-0.3 if m & 1 else 0.3)
    # positions stay in the half-open box
    L = np.asarray(b.L)[:, None]
    assert np.all(out[:3] >= -L / 2) and np.all(out[:3] < L / 2)


@pytest.mark.parametrize("m", [6, 8, 14])
def test_shear_symmetric_mappings_commute_with_the_sheared_dynamics(m):
    """(x, y) -> (-x, -y) and z -> -z are symmetries of planar shear in x
    with gradient in y (SLLOD with Lees-Edwards images), so running the
    mapped state gives the mapped trajectory: map(evolve(G)) =
    evolve(map(G)) at gamma = 0.1 after 60 steps."""
    N = 256
    b = bulk(N)
    st = inputs.jittered_states(N, 1, seed=7, amp=0.1)[0]
    st[3:] = np.random.default_rng(3).standard_normal((3, N)) * np.sqrt(0.722)
    mapped, am = oracle.apply_mapping(b, m, st, alpha=0.05)
    s1, a1, d1, _ = oracle.trajectory(b, st, 60, gamma=0.1, alpha=0.05)
    s2, a2, d2, _ = oracle.trajectory(b, mapped, 60, gamma=0.1, alpha=am)
    ms1, _ = oracle.apply_mapping(b, m, s1, alpha=a1)
    L = np.asarray(b.L)[:, None]
    dx = s2[:3] - ms1[:3]
    # positions are compared modulo the periodic (Lees-Edwards) images
    dx[1] -= L[1] * np.rint(dx[1] / L[1])
    dx[0] -= L[0] * np.rint(dx[0] / L[0])
    dx[2] -= L[2] * np.rint(dx[2] / L[2])
    assert np.abs(dx).max() < 1e-8
    assert np.abs(s2[3:] - ms1[3:]).max() < 1e-8
    assert a2 == pytest.approx(a1, abs=1e-10)


def test_mapping_sets_closed_under_a_reflection_cancel_omega():
    """Sets of mapping codes closed under the x-reflection (m -> m ^ 2), such
    as all 32 codes or the 8 of Eq. 3 with and without the z-mirror, give
    sum_m Omega(0) = 0 and sum_m B(0) = 0 in every group, to rounding."""
    N = 256
    b = bulk(N)
    ms = inputs.jittered_states(N, 2, seed=21, amp=0.1)
    ms[:, 3:] = np.random.default_rng(8).standard_normal((2, 3, N))
    for mask in (0xFFFFFFFF, 0x0F0F, 0xFFFF):
        B, Om = oracle.daughters(b, ms, np.zeros(2), 1e-2, 2, mapping_mask=mask)
        M = bin(mask).count("1")
        for g in range(2):
            o = Om[g * M:(g + 1) * M]
            assert abs(o.sum()) <= 1e-12 * np.abs(o).sum(), hex(mask)
            assert abs(B[g * M:(g + 1) * M, 0].sum()) <= 1e-12 * np.abs(B[g * M:(g + 1) * M, 0]).sum()
