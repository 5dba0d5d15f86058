"""Pins of the oracle's equilibrium friction coefficient xi_0 (Eq. 12 by the
equilibrium method of the paper's references: the generalised Langevin
relation between the wall's force on the fluid and the slip velocity) against
a process whose friction kernel is known exactly.

The process: a slab velocity u driven only by the wall's force F = -z, with
the Maxwell memory kernel zeta(t) = (zeta_0/tau) exp(-t/tau) in its Markovian
embedding
    du = -z dt,   dz = (zeta_0/tau u - z/tau) dt + sqrt(2 kT zeta_0)/tau dW,
whose stationary covariance is diag(kT, kT zeta_0/tau) (Lyapunov equation)
and whose correlations are <x(t) x(0)^T> = expm(A t) Sigma.  With the wall at
rest the slip is dv = -u, so F(t) = int_0^t zeta(t - s) dv(s) ds + R(t): the
estimator must return zeta_0 (and tau_M = tau for the Maxwell fit)."""
import numpy as np
import pytest

from oracle import reduce as orr

scipy_linalg = pytest.importorskip("scipy.linalg")

ZETA0, TAU, KT = 5.0, 0.2, 1.0
A_MAT = np.array([[0.0, -1.0], [ZETA0 / TAU, -1.0 / TAU]])
SIGMA = np.diag([KT, KT * ZETA0 / TAU])


def test_lyapunov_stationary_covariance():
    noise = np.diag([0.0, 2.0 * KT * ZETA0 / TAU ** 2])
    assert np.allclose(A_MAT @ SIGMA + SIGMA @ A_MAT.T + noise, 0.0, atol=1e-12)


def exact_correlations(ds, max_lag):
    """C_dvF(k ds) = <dv(0) F(t)> = <u(0) z(t)>, C_dvdv = <u(0) u(t)>."""
    c_dvf, c_dvdv = [], []
    for k in range(max_lag + 1):
        C = scipy_linalg.expm(A_MAT * k * ds) @ SIGMA
        c_dvdv.append(C[0, 0])
        c_dvf.append(C[1, 0])
    return np.array(c_dvf), np.array(c_dvdv)


def test_exact_correlations_recover_the_maxwell_kernel():
    ds, max_lag = 0.005, 1200
    c_dvf, c_dvdv = exact_correlations(ds, max_lag)
    # velocity and force are uncorrelated at equal times (time reversal)
    assert abs(c_dvf[0]) < 1e-14
    s = np.linspace(0.1, 2.0, 20)
    out = orr.friction_from_correlations(c_dvf, c_dvdv, ds, 1.0, s)
    assert out["zeta0"] == pytest.approx(ZETA0, rel=1e-3)
    assert out["tau_m"] == pytest.approx(TAU, rel=1e-2)
    assert out["xi_ratio"] == pytest.approx(ZETA0, rel=1e-3)
    # per wall area
    out2 = orr.friction_from_correlations(c_dvf, c_dvdv, ds, 4.0, s)
    assert out2["xi0"] == pytest.approx(ZETA0 / 4.0, rel=1e-3)
    # the Laplace ratio itself follows the Maxwell form
    assert np.allclose(out["zeta_s"], ZETA0 / (1.0 + s * TAU), rtol=2e-3)


def test_sampled_trajectories_recover_zeta0():
    """The same process sampled exactly in discrete time (64 trajectories,
    t = 100 each): the estimator on the series returns zeta_0 within its
    statistical error."""
    rng = np.random.default_rng(12)
    G, n, ds = 64, 5000, 0.02
    E = scipy_linalg.expm(A_MAT * ds)
    Q = SIGMA - E @ SIGMA @ E.T                       # covariance of one step's noise
    Lq = np.linalg.cholesky(Q)
    Ls = np.linalg.cholesky(SIGMA)
    x = Ls @ rng.standard_normal((2, G))
    u = np.empty((G, n))
    z = np.empty((G, n))
    for k in range(n):
        u[:, k], z[:, k] = x[0], x[1]
        x = E @ x + Lq @ rng.standard_normal((2, G))
    dv, F = -u, -z
    c_dvf = orr.cross_correlation(dv, F, 200)
    c_dvdv = orr.cross_correlation(dv, dv, 200)
    out = orr.friction_from_correlations(c_dvf, c_dvdv, ds, 1.0, np.linspace(0.1, 2.0, 20))
    assert out["zeta0"] == pytest.approx(ZETA0, rel=0.1)


def test_slip_and_wall_force_from_the_confined_responses():
    """dv = inner wall layer velocity - adjacent fluid velocity, F = -A sigma_w,
    on responses built with known values."""
    ns, G, S, A, n_layer = 40, 2, 7, 3.5, 50
    rng = np.random.default_rng(1)
    ser = np.zeros((G, 2 + 2 * ns + 2, S))
    slabs = [3, 4]
    v_fluid = rng.standard_normal((G, S))
    v_wall = rng.standard_normal((G, S))
    sigma = rng.standard_normal((G, S))
    for wall in (0, 1):
        ser[:, wall] = sigma
        ser[:, 2 + 2 * ns + wall] = n_layer * v_wall
    for j, k in enumerate(slabs):
        ser[:, 2 + ns + k] = 10 + j
        ser[:, 2 + k] = (10 + j) * v_fluid
    dv, F = orr.slip_and_wall_force(ser, A, n_layer, slabs, 1, ns)
    assert np.allclose(dv, v_wall - v_fluid, rtol=1e-13)
    assert np.allclose(F, -A * sigma, rtol=1e-15)
    # cross_correlation: <a(t) b(t+k)> over rows and origins
    a = np.array([[1.0, 2.0, 3.0]])
    b = np.array([[4.0, 5.0, 6.0]])
    assert np.allclose(orr.cross_correlation(a, b, 2), [(4 + 10 + 18) / 3, (5 + 12) / 2, 6.0])
