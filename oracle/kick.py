"""Further mother states from one thermalised state by small random momentum
kicks, plain numpy (test infrastructure: only tests, the smoke check and the
benchmark's CPU baseline use this module).

The paper's thermalisation workflow (section on the computational set-up)
generates further initial conditions from a single equilibrated state by
adding a small random kick to the velocities; the dynamics is chaotic, so
the kicked copies decorrelate quickly while the thermodynamic state is
kept.  The paper fixes neither the distribution nor what is conserved; the
reading implemented here (and by the CUDA path, from the same definitions):

  * copy c adds to momentum component k of atom i the kick
        dp = kick * sqrt(m k_B T) * g,  g ~ N(0, 1)   (m = k_B = 1)
    with g from Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
    the 64-bit seed (low word first), counter (i, c, b, 0) for block b = 0, 1,
    and Box-Muller on the 53-bit uniforms u = top53(w_hi, w_lo) / 2^53 + 2^-54
    (top53: the high 53 bits of the 64-bit word w_hi w_lo) of the output
    word pairs (w0, w1) -> u_a and (w2, w3) -> u_b:
        (g_2b, g_2b+1) = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b),
    of which g_0, g_1, g_2 kick x, y, z;
  * every group of atoms (the bulk system: all atoms; the confined system:
    fluid, bottom wall, top wall) keeps its net momentum: the group mean of
    the kicks is removed;
  * with keep_energy, every group also keeps its kinetic energy: with q the
    momenta relative to the group mean pbar and q' the kicked ones, the
    result is pbar + lambda q', lambda = sqrt(sum |q|^2 / sum |q'|^2)
    (lambda = 1 when sum |q'|^2 = 0).

Positions are copied unchanged.  States are [6, N] (x, y, z, px, py, pz).
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57          # Philox-4x32 multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85          # Weyl key increments
MASK = 0xFFFFFFFF


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Ten rounds of Philox-4x32 on counters ctr [..., 4] (uint32) with the
    2-word key; returns [..., 4] uint32.  One round: with the products
    hi/lo of M0*c0 and M1*c2, the new counter is
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
    and the key is bumped by the Weyl increments between rounds."""
    c = [ctr[..., j].astype(np.uint64) for j in range(4)]
    k0, k1 = np.uint64(key[0] & MASK), np.uint64(key[1] & MASK)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    mask = np.uint64(MASK)
    for r in range(10):
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        if r < 9:
            k0 = (k0 + np.uint64(W0)) & mask
            k1 = (k1 + np.uint64(W1)) & mask
    return np.stack([x.astype(np.uint32) for x in c], axis=-1)


def uniform53(w_hi: np.ndarray, w_lo: np.ndarray) -> np.ndarray:
    """Uniform in (0, 1) from two 32-bit words: the top 53 bits of
    w_hi * 2^32 + w_lo, plus half a step (never 0, never 1)."""
    v = (w_hi.astype(np.uint64) << np.uint64(32)) | w_lo.astype(np.uint64)
    return (v >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 + 2.0 ** -54


def gaussians(n_atoms: int, copy: int, seed: int) -> np.ndarray:
    """The three standard normal numbers [3, N] that kick atom i of copy c."""
    key = (seed & MASK, (seed >> 32) & MASK)
    g = np.empty((4, n_atoms))
    for b in (0, 1):
        ctr = np.zeros((n_atoms, 4), dtype=np.uint32)
        ctr[:, 0] = np.arange(n_atoms, dtype=np.uint32)
        ctr[:, 1] = copy
        ctr[:, 2] = b
        w = philox4x32_10(ctr, key)
        ua = uniform53(w[:, 0], w[:, 1])
        ub = uniform53(w[:, 2], w[:, 3])
        r = np.sqrt(-2.0 * np.log(ua))
        g[2 * b] = r * np.cos(2.0 * np.pi * ub)
        g[2 * b + 1] = r * np.sin(2.0 * np.pi * ub)
    return g[:3]


def kick_states(state: np.ndarray, n_copies: int, kick: float, T: float, seed: int,
                types: np.ndarray | None = None, keep_energy: bool = True) -> np.ndarray:
    """[n_copies, 6, N] kicked copies of one state [6, N] (see the module
    docstring for the definition)."""
    state = np.asarray(state, dtype=np.float64)
    N = state.shape[1]
    grp = np.zeros(N, dtype=np.int64) if types is None else np.asarray(types, dtype=np.int64)
    out = np.repeat(state[None], n_copies, axis=0)
    p = state[3:]
    for c in range(n_copies):
        dp = kick * np.sqrt(T) * gaussians(N, c, seed)
        pn = np.empty_like(p)
        for gi in np.unique(grp):
            sel = grp == gi
            pbar = p[:, sel].mean(axis=1, keepdims=True)
            q = p[:, sel] - pbar
            qk = q + (dp[:, sel] - dp[:, sel].mean(axis=1, keepdims=True))
            lam = 1.0
            if keep_energy:
                s_new = np.sum(qk * qk)
                lam = np.sqrt(np.sum(q * q) / s_new) if s_new > 0 else 1.0
            pn[:, sel] = pbar + lam * qk
        out[c, 3:] = pn
    return out
