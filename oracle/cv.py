"""Learned control variate for the TTCF estimator, plain numpy in FP64.

TEST INFRASTRUCTURE (see the package docstring).  The paper has no learned
part; this is the oracle of the CUDA control-variate kernels.  What it
computes (the readings are stated in the repository's design notes):

Features of a mapped mother state (32 numbers): kinetic and configurational
pressure tensors (6 + 6: xx yy zz xy xz yz), U/N, K/N with K = sum p^2 / 2,
the Nose-Hoover alpha, P_xy^2, and for q = 1..4 the cosine and sine modes
over 40 slabs in y of the density, (1/N) sum_i cs(2 pi q (k_i + 1/2) / 40),
and of the x momentum, (1/N) sum_i p_x,i cs(...), with k_i the slab of atom i.

Target of daughter d: z_d = Omega_d * I_d(t_end) / gamma, I_d the trapezoid
integral of B_d = P_xy.  Group value y_g = -(1/M) sum_m z_{g,m}, the group's
TTCF viscosity at t_end (Eq. 1, 7, 8; <B(0)> = 0 with all four mappings).

Network f: 32 -> 128 -> 128 -> 1, tanh hidden units, mean-squared loss;
parameters (flat, in this order) W1[128][32], b1[128], W2[128][128], b2[128],
W3[128], b3.  The GPU keeps FP32 master weights and computes with their BF16
rounding; ``bf16`` reproduces that rounding (nearest, ties to even).

Control-variate estimator over an evaluation set D of groups and an
independent auxiliary set M of mother states (features only):
    eta_cv = mean_D(y - c h) + c mean_M(h),  h_g = -(1/M) sum_m f(x_{g,m})
unbiased for any fixed network and c; its variance is
    Var_D(y - c h)/|D| + c^2 Var_M(h)/|M|.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 32
HIDDEN = 128
N_SLABS = 40
N_MODES = 4
N_PARAMS = HIDDEN * N_FEAT + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


# ------------------------------------------------------------ features --
def raw_features(b, state: np.ndarray) -> np.ndarray:
    """30 unmapped features of a state [6, N] (alpha is added by mapped_features):
    K_ab (6), W_ab (6) (virial sums, not divided by V), U, sum p^2,
    density modes (8), x-momentum modes (8)."""
    from .core import forces
    s = np.asarray(state, dtype=np.float64)
    N = s.shape[1]
    p = s[3:]
    K = np.array([np.sum(p[0] * p[0]), np.sum(p[1] * p[1]), np.sum(p[2] * p[2]),
                  np.sum(p[0] * p[1]), np.sum(p[0] * p[2]), np.sum(p[1] * p[2])])
    _, W, U = forces(b, s, 0.0)
    Ly = b.L[1]
    k = np.floor((s[1] + 0.5 * Ly) / Ly * N_SLABS)
    k = np.clip(k, 0, N_SLABS - 1)
    dens, mom = [], []
    for q in range(1, N_MODES + 1):
        ang = 2.0 * np.pi * q * (k + 0.5) / N_SLABS
        c, sn = np.cos(ang), np.sin(ang)
        dens += [np.sum(c) / N, np.sum(sn) / N]
        mom += [np.sum(p[0] * c) / N, np.sum(p[0] * sn) / N]
    return np.concatenate([K, W, [U, np.sum(p * p)], dens, mom])


def mapped_features(raw: np.ndarray, alpha: float, m: int, N: int, V: float,
                    reset_alpha: bool = False) -> np.ndarray:
    """The 32 features of mapping m (Eq. 3) from the unmapped raw features:
    x-reflections (m = 2, 3) negate the xy and xz stresses; momentum
    reversal (m = 1) and x-reflection with p_x flip (m = 2) negate the
    x-momentum modes; the time-reversing mappings (1, 3) negate alpha."""
    K, W, U, K2 = raw[0:6], raw[6:12], raw[12], raw[13]
    dens, mom = raw[14:22], raw[22:30]
    sxy = -1.0 if m in (2, 3) else 1.0
    sm = -1.0 if m in (1, 2) else 1.0
    sa = -1.0 if m in (1, 3) else 1.0
    sig = np.array([1, 1, 1, sxy, sxy, 1.0])
    PK = K * sig / V
    PC = W * sig / V
    pxy = PK[3] + PC[3]
    a = 0.0 if reset_alpha else sa * alpha
    return np.concatenate([PK, PC, [U / N, 0.5 * K2 / N, a, pxy * pxy], dens, sm * mom])


def targets(B: np.ndarray, Omega: np.ndarray, gamma, ds: float) -> np.ndarray:
    """z_d = Omega_d * trapezoid(B_d) / gamma (gamma scalar or per daughter)."""
    I = ds * (0.5 * (B[:, 0] + B[:, -1]) + B[:, 1:-1].sum(axis=1))
    return Omega * I / np.asarray(gamma, dtype=np.float64)


# ------------------------------------------------------------- network --
def unpack(theta: np.ndarray):
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = t[o:o + HIDDEN * N_FEAT].reshape(HIDDEN, N_FEAT); o += HIDDEN * N_FEAT
    b1 = t[o:o + HIDDEN]; o += HIDDEN
    W2 = t[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = t[o:o + HIDDEN]; o += HIDDEN
    W3 = t[o:o + HIDDEN]; o += HIDDEN
    b3 = t[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta: np.ndarray, X: np.ndarray):
    """Network output [n] and the activations needed by backward."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.tanh(X @ W1.T + b1)
    H2 = np.tanh(H1 @ W2.T + b2)
    out = H2 @ W3 + b3
    return out, (X, H1, H2)


def backward(theta: np.ndarray, X: np.ndarray, y: np.ndarray):
    """Loss (1/n) sum (f(x) - y)^2 and its gradient (flat, like theta)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    out, (X, H1, H2) = forward(theta, X)
    n = X.shape[0]
    r = out - np.asarray(y, dtype=np.float64)
    loss = np.mean(r * r)
    dout = 2.0 * r / n
    gW3 = H2.T @ dout
    gb3 = dout.sum()
    dA2 = np.outer(dout, W3) * (1.0 - H2 * H2)
    gW2 = dA2.T @ H1
    gb2 = dA2.sum(axis=0)
    dA1 = (dA2 @ W2) * (1.0 - H1 * H1)
    gW1 = dA1.T @ X
    gb1 = dA1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; t >= 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------ estimator --
def fit_c(y: np.ndarray, h: np.ndarray) -> float:
    """Variance-minimising coefficient Cov(y, h) / Var(h)."""
    y = np.asarray(y, dtype=np.float64); h = np.asarray(h, dtype=np.float64)
    hv = h - h.mean()
    return float(np.dot(y - y.mean(), hv) / np.dot(hv, hv))


def cv_estimate(y_D, h_D, h_M, c: float):
    """(eta_cv, se_cv, eta_plain, se_plain) for one c."""
    y_D = np.asarray(y_D, dtype=np.float64)
    h_D = np.asarray(h_D, dtype=np.float64)
    h_M = np.asarray(h_M, dtype=np.float64)
    nD, nM = len(y_D), len(h_M)
    r = y_D - c * h_D
    eta = r.mean() + c * h_M.mean()
    se = np.sqrt(r.var(ddof=1) / nD + c * c * h_M.var(ddof=1) / nM)
    return float(eta), float(se), float(y_D.mean()), float(y_D.std(ddof=1) / np.sqrt(nD))
