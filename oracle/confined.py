"""ctypes wrapper of the confined-system oracle ttcf_confined.c (Example 2;
test infrastructure).  Units: sigma = epsilon = m = k_B = 1."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .core import lib as _lib_bulk

N_SLAB = 40
# responses per sample: wall stress (bottom, top), 40 slab sums of fluid p_x,
# 40 slab counts, inner-layer p_x sums (bottom, top)
N_OBS = 2 + 2 * N_SLAB + 2
_configured = False


class _Conf(C.Structure):
    _fields_ = [("n", C.c_int), ("nslab", C.c_int), ("use_cells", C.c_int), ("pad_", C.c_int),
                ("L", C.c_double * 3), ("dt", C.c_double), ("Tw", C.c_double), ("Q", C.c_double),
                ("g", C.c_double), ("k", C.c_double), ("rc", C.c_double), ("c_ff", C.c_double),
                ("c_wf", C.c_double), ("c_ww", C.c_double), ("vwall", C.c_double),
                ("ww_on", C.c_int), ("pad2_", C.c_int)]


def lib():
    global _configured
    L = _lib_bulk()
    if not _configured:
        dp, ip, cp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(_Conf)
        L.orc_conf_forces.argtypes = [cp, ip, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_conf_forces.restype = C.c_int
        L.orc_conf_trajectory.argtypes = [cp, ip, dp, dp, dp, C.c_int, dp]
        L.orc_conf_trajectory.restype = C.c_int
        L.orc_conf_mother.argtypes = [cp, ip, dp, dp, C.c_int, C.c_int, C.c_int, dp, dp]
        L.orc_conf_mother.restype = C.c_int
        L.orc_conf_map.argtypes = [cp, C.c_int, dp, dp, C.c_double, C.c_int, dp, dp, dp]
        L.orc_conf_map.restype = None
        L.orc_conf_daughter.argtypes = [cp, ip, dp, dp, C.c_double, C.c_int, C.c_int, C.c_int,
                                        C.c_int, dp, dp, dp]
        L.orc_conf_daughter.restype = C.c_int
        L.orc_conf_daughters.argtypes = [cp, ip, C.c_int, dp, dp, dp, C.c_int, C.c_int, dp, dp, C.c_int]
        L.orc_conf_daughters.restype = C.c_int
        _configured = True
    return L


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int))


@dataclass
class Confined:
    """Example 2: LJ with wetting parameters (Eq. 9), tethered walls with a
    wall-only Nose-Hoover thermostat and sliding lattices (Eq. 10)."""
    types: np.ndarray
    box: tuple
    dt: float = 0.005
    Tw: float = 1.0
    tau_T: float = 0.25
    k: float = 150.0
    rc: float = 2.5
    c_ff: float = 1.2
    c_wf: float = 0.6325
    c_ww: float = 1.0          # wall-wall (not given in the paper: plain LJ)
    ww_on: bool = True         # False: the tethers alone hold the walls
    vwall: float = 0.0
    use_cells: bool = True
    nslab: int = N_SLAB

    @property
    def n(self) -> int:
        return len(self.types)

    @property
    def n_wall(self) -> int:
        return int(np.sum(self.types != 0))

    @property
    def g(self) -> float:
        return 3.0 * self.n_wall

    @property
    def Q(self) -> float:
        return self.g * self.Tw * self.tau_T ** 2

    @property
    def area(self) -> float:
        return float(self.box[0] * self.box[2])

    def c(self, vwall=None) -> _Conf:
        s = _Conf()
        s.n, s.nslab, s.use_cells = self.n, self.nslab, 1 if self.use_cells else 0
        for d in range(3):
            s.L[d] = float(self.box[d])
        s.dt, s.Tw, s.Q, s.g, s.k, s.rc = self.dt, self.Tw, self.Q, self.g, self.k, self.rc
        s.c_ff, s.c_wf, s.c_ww = self.c_ff, self.c_wf, self.c_ww
        s.ww_on = 1 if self.ww_on else 0
        s.vwall = self.vwall if vwall is None else vwall
        return s

    @property
    def t(self) -> np.ndarray:
        return np.ascontiguousarray(self.types, dtype=np.int32)


def forces(sys: Confined, state, lattice, cells=None):
    """(F [3, N], U_pair, U_tether, fluid x force on [bottom, top] wall)."""
    s = np.ascontiguousarray(state, np.float64)
    lt = np.ascontiguousarray(lattice, np.float64)
    F = np.zeros((3, sys.n))
    U = np.zeros(2)
    sw = np.zeros(2)
    c = sys.c()
    if cells is not None:
        c.use_cells = 1 if cells else 0
    rc = lib().orc_conf_forces(C.byref(c), _ip(sys.t), _p(s[0]), _p(s[1]), _p(s[2]), _p(lt[0]),
                               _p(lt[1]), _p(lt[2]), _p(F[0]), _p(F[1]), _p(F[2]), _p(U), _p(sw))
    if rc:
        raise RuntimeError(f"confined forces failed ({rc})")
    return F, U[0], U[1], sw


def trajectory(sys: Confined, state, lattice, n_steps: int, alpha: float = 0.0):
    """obs columns: K, U_pair, U_tether, alpha, xi, H_ext, P_lattice."""
    s = np.array(state, np.float64, order="C")
    lt = np.array(lattice, np.float64, order="C")
    a = C.c_double(alpha)
    obs = np.zeros((n_steps + 1, 7))
    if lib().orc_conf_trajectory(C.byref(sys.c()), _ip(sys.t), _p(s), _p(lt), C.byref(a),
                                 int(n_steps), _p(obs)):
        raise RuntimeError("confined trajectory failed")
    return s, lt, a.value, obs


def mother(sys: Confined, init, lattice, n_eq: int, n_states: int, spacing: int):
    s = np.ascontiguousarray(init, np.float64)
    lt = np.ascontiguousarray(lattice, np.float64)
    out = np.zeros((n_states, 6, sys.n))
    al = np.zeros(n_states)
    if lib().orc_conf_mother(C.byref(sys.c()), _ip(sys.t), _p(s), _p(lt), int(n_eq), int(n_states),
                             int(spacing), _p(out), _p(al)):
        raise RuntimeError("confined mother failed")
    return out, al


def apply_mapping(sys: Confined, m: int, state, lattice, alpha: float = 0.0):
    s = np.ascontiguousarray(state, np.float64)
    lt = np.ascontiguousarray(lattice, np.float64)
    out, lo = np.empty_like(s), np.empty_like(lt)
    a = C.c_double()
    lib().orc_conf_map(C.byref(sys.c()), int(m), _p(s), _p(lt), float(alpha), 0, _p(out), _p(lo),
                       C.byref(a))
    return out, lo, a.value


def daughter(sys: Confined, mother_state, lattice, mother_alpha, m, n_steps, sample_every=1):
    """(B [S, 2 + 2 nslab + 2], Omega, final state)."""
    s = np.ascontiguousarray(mother_state, np.float64)
    lt = np.ascontiguousarray(lattice, np.float64)
    S = n_steps // sample_every + 1
    B = np.zeros((S, 2 + 2 * sys.nslab + 2))
    om = C.c_double()
    fin = np.zeros((6, sys.n))
    if lib().orc_conf_daughter(C.byref(sys.c()), _ip(sys.t), _p(s), _p(lt), float(mother_alpha),
                               int(m), 0, int(n_steps), int(sample_every), _p(B), C.byref(om),
                               _p(fin)):
        raise RuntimeError("confined daughter failed")
    return B, om.value, fin


def daughters(sys: Confined, mothers, lattice, alphas, n_steps, sample_every=1, n_threads=None):
    """B [4G, S, 2 + 2 nslab + 2], Omega [4G]; daughter d = 4 g + m."""
    ms = np.ascontiguousarray(mothers, np.float64)
    lt = np.ascontiguousarray(lattice, np.float64)
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(alphas, np.float64), (ms.shape[0],)))
    G = ms.shape[0]
    S = n_steps // sample_every + 1
    B = np.zeros((4 * G, S, 2 + 2 * sys.nslab + 2))
    Om = np.zeros(4 * G)
    nt = n_threads or os.cpu_count() or 1
    if lib().orc_conf_daughters(C.byref(sys.c()), _ip(sys.t), G, _p(ms), _p(lt), _p(al), int(n_steps),
                                int(sample_every), _p(B), _p(Om), int(nt)):
        raise RuntimeError("confined daughters failed")
    return B, Om


def inner_layer(types, lattice, wall: int, tol: float = 0.1) -> np.ndarray:
    """Indices of the innermost layer of wall 0 (bottom, type 1) or 1 (top,
    type 2): the wall's atoms whose tether site lies within tol in y of the
    wall's site plane nearest the channel."""
    t = np.asarray(types)
    yl = np.asarray(lattice)[1]
    sel = t == (1 if wall == 0 else 2)
    if wall == 0:
        return np.nonzero(sel & (yl >= yl[sel].max() - tol))[0]
    return np.nonzero(sel & (yl <= yl[sel].min() + tol))[0]
