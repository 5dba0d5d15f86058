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


# ---------------------------------------------------------------- confined --
# Example 2 geometry: a fluid layer between two FCC(111) walls lying in the
# xz plane, with x along a close-packed row so that x -> -x maps each wall
# onto itself (the x-reflection mappings of Eq. 3 then map the ensemble onto
# itself).  Walls at number density RHO_WALL, channel width H_CHANNEL
# between the innermost wall layers, fluid on a cubic lattice at RHO_FLUID.
RHO_WALL = 0.8
RHO_FLUID = 0.8
H_CHANNEL = 10.0
T_WALL = 1.0
DT_CONFINED = 0.005

FLUID, WALL_BOTTOM, WALL_TOP = 0, 1, 2


def confined_system(nx: int = 25, nz: int = 28, layers: int = 3, seed: int = BASE_SEED,
                    rho_fluid: float = RHO_FLUID, h: float = H_CHANNEL, T: float = T_WALL):
    """Initial state of the confined system.

    Returns a dict with ``state`` [6, N] (x y z px py pz, x and z in the
    centred periodic box, y non-periodic), ``types`` [N] int32 (0 fluid,
    1 bottom wall, 2 top wall), ``lattice`` [3, N] tether sites (walls; the
    fluid rows repeat the positions), ``box`` (Lx, Ly, Lz) with Ly the slab
    extent used for the velocity profile, and the counts.  nz must be even."""
    if nz % 2:
        raise ValueError("nz must be even")
    a = (4.0 / RHO_WALL) ** (1.0 / 3.0)
    d = a / np.sqrt(2.0)                  # in-plane nearest-neighbour spacing
    dz = d * np.sqrt(3.0) / 2.0           # row spacing of the triangular layer
    dy = a / np.sqrt(3.0)                 # (111) layer spacing
    Lx, Lz = nx * d, nz * dz
    walls = []
    for side, sgn in ((WALL_BOTTOM, -1.0), (WALL_TOP, 1.0)):
        for lay in range(layers):
            y = sgn * (0.5 * h + lay * dy)
            for r in range(nz):
                # ABC stacking: x offset alternates by row and shifts by layer;
                # z shifts by a third of a row per layer
                phase = 0.5 * ((r + lay) % 2)
                z = (r + lay / 3.0) * dz - 0.5 * Lz
                for i in range(nx):
                    x = (i + phase) * d - 0.5 * Lx
                    walls.append((x, y, z, side))
    W = np.array(walls)
    W[:, 2] -= Lz * np.floor((W[:, 2] + 0.5 * Lz) / Lz)
    # fluid on a cubic lattice filling |y| <= h/2 - 1 (one diameter from
    # the innermost wall layer)
    sp = (1.0 / rho_fluid) ** (1.0 / 3.0)
    fx, fz = int(Lx / sp), int(Lz / sp)
    ymax = 0.5 * h - 1.0
    fy = int(2 * ymax / sp) + 1
    gx = (np.arange(fx) + 0.5) * (Lx / fx) - 0.5 * Lx
    gz = (np.arange(fz) + 0.5) * (Lz / fz) - 0.5 * Lz
    gy = np.linspace(-ymax, ymax, fy)
    F = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), axis=-1).reshape(-1, 3)
    n_f, n_w = len(F), len(W)
    N = n_f + n_w
    pos = np.concatenate([F, W[:, :3]]).T
    types = np.concatenate([np.zeros(n_f, np.int32), W[:, 3].astype(np.int32)])
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((3, N)) * np.sqrt(T)
    for t in (FLUID, WALL_BOTTOM, WALL_TOP):
        sel = types == t
        p[:, sel] -= p[:, sel].mean(axis=1, keepdims=True)
    state = np.ascontiguousarray(np.concatenate([pos, p]))
    Ly = 2.0 * (0.5 * h + (layers - 1) * dy + 1.0)
    return {"state": state, "types": types, "lattice": np.ascontiguousarray(pos.copy()),
            "box": np.array([Lx, Ly, Lz]), "n_fluid": n_f, "n_wall": n_w, "h": h,
            "layer_spacing": dy, "row_spacing": d}
