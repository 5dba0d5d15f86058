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


def friction(resp_obs, gamma: float, Ly: float, h: float, wall: int, nslab: int = 40,
             estimator: str = "ttcf") -> dict:
    """Slip velocity and friction coefficient of Eq. 12 at one wall from the
    confined responses (resp_obs[o] = responses of observable o):
    v(t) = sum_k <P_k> / sum_k <n_k> over the slabs adjacent to the wall,
    slip = v - s_w gamma h / 2, xi = <sigma_w> / slip (sigma_w: x force of
    the fluid on the wall per area; s_w = -1 bottom, +1 top)."""
    ks = adjacent_slabs(Ly, h, wall, nslab)
    P = sum(resp_obs[2 + k][estimator] for k in ks)
    n = sum(resp_obs[2 + nslab + k][estimator] for k in ks)
    sw = 1.0 if wall == 1 else -1.0
    slip = P / n - sw * gamma * 0.5 * h
    sigma = resp_obs[wall][estimator]
    with np.errstate(divide="ignore", invalid="ignore"):
        xi = sigma / slip
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
