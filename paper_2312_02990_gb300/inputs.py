"""Seeded synthetic inputs for the TTCF daughter ensemble.

This module is shared by the CUDA path, the CPU oracle and the tests.  It
holds no arithmetic of the TTCF method itself: it only lays atoms on a
face-centred-cubic lattice and draws Maxwell-Boltzmann momenta, which is the
starting point of the equilibrium mother trajectory (Section "Mathematical
Framework" and Algorithm 2, "initialize system").  The mother trajectory and
everything after it are computed by each side with its own code.

State layout used everywhere: a C-contiguous float64 array ``[6, N]`` holding
rows x, y, z, px, py, pz (peculiar momenta, unit mass), positions in the
centred box [-L/2, L/2).
"""
from __future__ import annotations

import numpy as np

# Reduced units: sigma = epsilon = m = k_B = 1 (Example 1 state point).
RHO_TRIPLE = 0.8442
T_TRIPLE = 0.722
DT_BULK = 0.0025
BASE_SEED = 20231205


def fcc_cells_for(n_atoms: int) -> int:
    """Number of FCC unit cells per side for an FCC-exact atom count 4 n^3."""
    n = int(round((n_atoms / 4) ** (1.0 / 3.0)))
    if 4 * n ** 3 != n_atoms:
        raise ValueError(f"n_atoms={n_atoms} is not 4*n^3")
    return n


def bulk_box(n_atoms: int, rho: float = RHO_TRIPLE) -> np.ndarray:
    """Cubic box edge lengths [Lx, Ly, Lz] for N atoms at number density rho."""
    L = (n_atoms / rho) ** (1.0 / 3.0)
    return np.array([L, L, L], dtype=np.float64)


def fcc_lattice(n_atoms: int, rho: float = RHO_TRIPLE) -> np.ndarray:
    """FCC positions [3, N] in the centred cubic box, shifted by a/4 so that
    no atom sits on a box face."""
    n = fcc_cells_for(n_atoms)
    L = bulk_box(n_atoms, rho)[0]
    a = L / n
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n),
                                 indexing="ij"), axis=-1).reshape(-1, 3)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    pos = pos - L / 2 + a / 4
    return np.ascontiguousarray(pos.T)


def maxwell_momenta(n_atoms: int, T: float, seed: int, dof: int | None = None) -> np.ndarray:
    """Gaussian momenta [3, N] with zero total momentum, rescaled so that
    sum p^2 = dof * T exactly (dof defaults to 3N)."""
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((3, n_atoms)) * np.sqrt(T)
    p -= p.mean(axis=1, keepdims=True)
    dof = 3 * n_atoms if dof is None else dof
    p *= np.sqrt(dof * T / np.sum(p * p))
    return p


def initial_state(n_atoms: int, seed: int, T: float = T_TRIPLE,
                  rho: float = RHO_TRIPLE) -> np.ndarray:
    """Lattice + Maxwell state [6, N] (x, y, z, px, py, pz)."""
    s = np.empty((6, n_atoms), dtype=np.float64)
    s[:3] = fcc_lattice(n_atoms, rho)
    s[3:] = maxwell_momenta(n_atoms, T, seed)
    return np.ascontiguousarray(s)


def jittered_states(n_atoms: int, n_states: int, seed: int, amp: float = 0.05,
                    T: float = T_TRIPLE, rho: float = RHO_TRIPLE) -> np.ndarray:
    """[n_states, 6, N] lattice states with small uniform position jitter and
    independent Maxwell momenta.  Used where a test needs many distinct
    states without running an equilibrium trajectory (force and mapping
    parity); they are not equilibrium samples."""
    rng = np.random.default_rng(seed)
    L = bulk_box(n_atoms, rho)[0]
    out = np.empty((n_states, 6, n_atoms), dtype=np.float64)
    base = fcc_lattice(n_atoms, rho)
    for k in range(n_states):
        pos = base + rng.uniform(-amp, amp, size=base.shape)
        pos = pos - L * np.floor((pos + L / 2) / L)
        out[k, :3] = pos
        out[k, 3:] = maxwell_momenta(n_atoms, T, seed * 1000003 + k)
    return out
