"""Ensemble averages of the TTCF method, plain numpy (test infrastructure).

Inputs are per-daughter responses ``B[D, S]`` (sample s at time s*ds) and
dissipation values ``Omega[D]``, daughters ordered ``d = g*M + k`` with M
mapped daughters per mother state g.

    integrand   <Omega(0) B(s)>          = (1/D) sum_d Omega_d B_d(s)       Eq. 2
    TTCF        <B(t)> = <B(0)> + int_0^t <Omega(0) B(s)> ds                Eq. 1
    corrected   <Omega(0)B(s)> - <Omega(0)><B(s)>                           Eq. 4
    DAV         <B(t)> = (1/D) sum_d B_d(t)                  direct average
    viscosity   eta(t) = -<P_xy(t)>/gamma                    Eq. 8
    equilibrium <B(t)B(t+k)> over trajectories and time origins, and the
                Green-Kubo integral (V/k_BT) int <P_xy(0)P_xy(t)> dt
                (Eq. 8 at zero field; the mother-side correlations of Fig. 7)

The integral is the trapezoid rule on the sample grid.  Standard errors are
taken over mother groups (each group's mean over its M mapped daughters is
one independent sample), SE = std_g / sqrt(G) with ddof = 1; the mappings
make the group means of B(0) identical (zero), so the DAV standard error is
zero at t = 0, as the paper observes for Fig. 8.
"""
from __future__ import annotations

import numpy as np


def _cumtrapz(y: np.ndarray, dx: float) -> np.ndarray:
    """Cumulative trapezoid along the last axis, starting at 0."""
    out = np.zeros_like(y)
    out[..., 1:] = np.cumsum(0.5 * dx * (y[..., 1:] + y[..., :-1]), axis=-1)
    return out


def _se(groups: np.ndarray) -> np.ndarray:
    G = groups.shape[0]
    if G < 2:
        return np.full(groups.shape[1:], np.nan)
    return groups.std(axis=0, ddof=1) / np.sqrt(G)


def responses(B: np.ndarray, Omega: np.ndarray, M: int, ds: float,
              corrected: bool = False) -> dict:
    """Per-time ensemble means and group standard errors."""
    B = np.asarray(B, dtype=np.float64)
    Om = np.asarray(Omega, dtype=np.float64)
    D, S = B.shape
    G = D // M
    Bg = B.reshape(G, M, S)
    Og = Om.reshape(G, M)
    Y = np.einsum("gm,gms->gs", Og, Bg) / M      # group mean of Omega*B
    Dg = Bg.mean(axis=1)                         # group mean of B
    Jg = Dg[:, :1] + _cumtrapz(Y, ds)            # group TTCF estimate
    corr = Y.mean(axis=0)
    dav = Dg.mean(axis=0)
    om_mean = Og.mean()
    if corrected:
        corr_c = corr - om_mean * dav
        ttcf = dav[0] + _cumtrapz(corr_c, ds)
    else:
        ttcf = Jg.mean(axis=0)
    return {
        "t": np.arange(S) * ds,
        "corr": corr, "corr_se": _se(Y),
        "dav": dav, "dav_se": _se(Dg),
        "ttcf": ttcf, "ttcf_se": _se(Jg),
        "omega_mean": om_mean,
        "dav_se_daughters": B.std(axis=0, ddof=1) / np.sqrt(D),
        "corr_se_daughters": (Om[:, None] * B).std(axis=0, ddof=1) / np.sqrt(D),
    }


def viscosity(resp: dict, gamma: float) -> dict:
    """Eq. 8 with the standard pressure tensor: eta = -<P_xy>/gamma."""
    return {
        "t": resp["t"],
        "eta_ttcf": -resp["ttcf"] / gamma, "eta_ttcf_se": resp["ttcf_se"] / abs(gamma),
        "eta_dav": -resp["dav"] / gamma, "eta_dav_se": resp["dav_se"] / abs(gamma),
    }


def adjacent_slabs(Ly: float, h: float, wall: int, nslab: int = 40, width: float = 1.0):
    """Slabs whose centres lie within `width` of the innermost layer of a
    wall, on the fluid side (wall 0: bottom at y = -h/2, 1: top at +h/2)."""
    w = Ly / nslab
    centres = -0.5 * Ly + (np.arange(nslab) + 0.5) * w
    if wall == 1:
        sel = (centres > 0.5 * h - width) & (centres < 0.5 * h)
    else:
        sel = (centres < -0.5 * h + width) & (centres > -0.5 * h)
    return np.nonzero(sel)[0]


def friction(resp_obs, Ly: float, h: float, wall: int, n_layer: int, nslab: int = 40,
             estimator: str = "ttcf") -> dict:
    """Slip velocity and friction coefficient of Eq. 12 at one wall from the
    confined responses (resp_obs[o] = responses of observable o), with the
    slip velocity as the paper defines it: the velocity of the innermost wall
    layer minus that of the outermost fluid layer,
        v_wall  = <sum of p_x over the wall's innermost layer> / n_layer
                  (observable 2 + 2 nslab + wall),
        v_fluid = sum_k <P_k> / sum_k <n_k> over the slabs adjacent to the
                  wall (each average a TTCF-able linear response; the ratio
                  is taken after averaging),
        slip    = v_wall - v_fluid,
        xi      = <F_x> / (A slip) = -<sigma_w> / slip,
    sigma_w being the x force of the fluid on the wall per area (the force
    of the wall on the fluid is its negative)."""
    ks = adjacent_slabs(Ly, h, wall, nslab)
    P = sum(resp_obs[2 + k][estimator] for k in ks)
    n = sum(resp_obs[2 + nslab + k][estimator] for k in ks)
    v_wall = resp_obs[2 + 2 * nslab + wall][estimator] / n_layer
    with np.errstate(divide="ignore", invalid="ignore"):
        slip = v_wall - P / n
        xi = -resp_obs[wall][estimator] / slip
    return {"slip": slip, "xi": xi, "slabs": ks}


def autocorrelation(B: np.ndarray, max_lag: int):
    """Time correlations of the series B[G, n] (G independent trajectories,
    one sample per step), averaged over trajectories and all time origins
    t = 0 .. n-1-k:
        acf[k]  = <B(t) B(t+k)>,
        acf2[k] = <(B(t)^2 - m2)(B(t+k)^2 - m2)>,   m2 = <B^2>,
    for lags k = 0 .. max_lag."""
    B = np.asarray(B, dtype=np.float64)
    if B.ndim == 1:
        B = B[None]
    n = B.shape[1]
    m2 = float(np.mean(B * B))
    acf = np.zeros(max_lag + 1)
    acf2 = np.zeros(max_lag + 1)
    for k in range(max_lag + 1):
        a, b = B[:, :n - k], B[:, k:]
        acf[k] = np.mean(a * b)
        acf2[k] = np.mean((a * a - m2) * (b * b - m2))
    return acf, acf2


def green_kubo(acf: np.ndarray, V: float, T: float, ds: float) -> np.ndarray:
    """Running Green-Kubo viscosity (V / k_B T) int_0^{k ds} <P_xy(0)P_xy(t)> dt
    by the trapezoid rule on the lag grid (Eq. 8 at zero field)."""
    return (V / T) * _cumtrapz(np.asarray(acf, dtype=np.float64), ds)


# ----------------------------------------------------------------------------
# Equilibrium friction coefficient xi_0 of Eq. 12 (<F_x> = xi_0 A <dv>), by
# the equilibrium method the paper takes from its references (Hansen, Todd
# and Daivis 2011; Varghese, Hansen and Todd 2021): along equilibrium
# trajectories (walls at rest) the force F(t) of the wall on the fluid next
# to it and the slip velocity dv(t) (innermost wall layer minus outermost
# fluid layer) obey a generalised Langevin relation F(t) = int_0^t
# zeta(t - u) dv(u) du + R(t) with a random force R uncorrelated with
# dv(0), so that
#     C_dvF(t) = <dv(0) F(t)> = int_0^t zeta(t - u) C_dvdv(u) du,
# and in the Laplace domain zeta~(s) = C~_dvF(s) / C~_dvdv(s).  The friction
# kernel is fitted with a Maxwell model zeta~(s) = zeta_0 / (1 + s tau_M),
# i.e. the straight line 1/zeta~(s) = 1/zeta_0 + (tau_M/zeta_0) s, and
# xi_0 = zeta_0 / A (the zero-frequency friction per wall area).
# ----------------------------------------------------------------------------
def cross_correlation(a: np.ndarray, b: np.ndarray, max_lag: int) -> np.ndarray:
    """<a(t) b(t+k)> over trajectories (rows) and time origins t = 0 ..
    n-1-k, for k = 0 .. max_lag."""
    a = np.atleast_2d(np.asarray(a, dtype=np.float64))
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    n = a.shape[1]
    return np.array([np.mean(a[:, :n - k] * b[:, k:]) for k in range(max_lag + 1)])


def laplace(c: np.ndarray, ds: float, s: float) -> float:
    """int_0^{t_max} exp(-s t) c(t) dt by the trapezoid rule on the lag grid."""
    t = np.arange(len(c)) * ds
    f = np.exp(-s * t) * np.asarray(c, dtype=np.float64)
    return float(ds * (f.sum() - 0.5 * (f[0] + f[-1])))


def friction_from_correlations(c_dvf, c_dvdv, ds: float, area: float, s_grid) -> dict:
    """xi_0 from the two equilibrium correlations: zeta~(s) on s_grid, the
    least-squares line through 1/zeta~(s), zeta_0 = 1 / intercept,
    tau_M = slope / intercept, xi_0 = zeta_0 / area; also the s = 0 ratio
    of the integrals (the unfitted estimate) as xi_ratio."""
    s_grid = np.asarray(s_grid, dtype=np.float64)
    zeta = np.array([laplace(c_dvf, ds, s) / laplace(c_dvdv, ds, s) for s in s_grid])
    slope, icpt = np.polyfit(s_grid, 1.0 / zeta, 1)
    z0 = 1.0 / icpt
    return {"xi0": z0 / area, "zeta0": z0, "tau_m": slope / icpt, "s": s_grid, "zeta_s": zeta,
            "xi_ratio": laplace(c_dvf, ds, 0.0) / laplace(c_dvdv, ds, 0.0) / area}


def slip_and_wall_force(series: np.ndarray, area: float, n_layer: int, slabs, wall: int,
                        nslab: int = 40):
    """dv(t) and F(t) of each trajectory from the confined responses
    series[G, n_obs, S]: dv = (inner wall layer p_x sum) / n_layer - (sum
    of the adjacent slabs' p_x) / (their fluid count), F = -A sigma_w (the
    wall's force on the fluid; sigma_w is the fluid's x force on the wall
    per area)."""
    ser = np.asarray(series, dtype=np.float64)
    P = ser[:, [2 + k for k in slabs]].sum(axis=1)
    n = ser[:, [2 + nslab + k for k in slabs]].sum(axis=1)
    dv = ser[:, 2 + 2 * nslab + wall] / n_layer - P / n
    F = -area * ser[:, wall]
    return dv, F


def friction_equilibrium(series, area: float, n_layer: int, slabs, wall: int, ds: float,
                         max_lag: int, s_grid, nslab: int = 40) -> dict:
    """xi_0 of one wall from equilibrium confined trajectories (see above)."""
    dv, F = slip_and_wall_force(series, area, n_layer, slabs, wall, nslab)
    c_dvf = cross_correlation(dv, F, max_lag)
    c_dvdv = cross_correlation(dv, dv, max_lag)
    out = friction_from_correlations(c_dvf, c_dvdv, ds, area, s_grid)
    out.update({"c_dvf": c_dvf, "c_dvdv": c_dvdv})
    return out
