"""ctypes wrapper of the FP64 C oracle ``ttcf_oracle.c`` (test infrastructure).

The shared object is compiled here with gcc (``build()``); nothing in this
package touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ttcf_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ttcf_confined.c")]
_SO = os.path.join(_HERE, "libttcf_oracle.so")
_lib = None

RC_WCA = 2.0 ** (1.0 / 6.0)


def build(force: bool = False) -> str:
    """Compile the oracle (portable flags: it builds on x86_64 and aarch64)."""
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-o", _SO, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


class _Bulk(C.Structure):
    _fields_ = [("n", C.c_int), ("use_cells", C.c_int), ("L", C.c_double * 3),
                ("dt", C.c_double), ("T", C.c_double), ("Q", C.c_double),
                ("g", C.c_double), ("rc", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp = C.POINTER(C.c_double)
        bp = C.POINTER(_Bulk)
        L.orc_wca.restype = C.c_double
        L.orc_wca.argtypes = [C.c_double, dp]
        for name in ("orc_forces_brute", "orc_forces_cells", "orc_forces"):
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = [bp, C.c_double, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_pressure.restype = C.c_int
        L.orc_pressure.argtypes = [bp, dp, C.c_double, dp, dp, dp]
        L.orc_state_forces.restype = C.c_int
        L.orc_state_forces.argtypes = [bp, dp, C.c_double, dp, dp, dp]
        L.orc_apply_mapping.restype = None
        L.orc_apply_mapping.argtypes = [bp, C.c_int, dp, C.c_double, C.c_int, dp, dp]
        L.orc_trajectory.restype = C.c_int
        L.orc_trajectory.argtypes = [bp, C.c_double, dp, dp, dp, C.c_int, dp]
        L.orc_mother.restype = C.c_int
        L.orc_mother.argtypes = [bp, dp, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp]
        L.orc_daughter.restype = C.c_int
        L.orc_daughter.argtypes = [bp, dp, C.c_double, C.c_int, C.c_int, C.c_double,
                                   C.c_int, C.c_int, dp, dp, dp, dp]
        L.orc_daughters.restype = C.c_int
        L.orc_daughters.argtypes = [bp, C.c_int, dp, dp, dp, C.c_uint, C.c_int, C.c_int,
                                    C.c_int, dp, dp, C.c_int]
        L.orc_trajectory_elong.restype = C.c_int
        L.orc_trajectory_elong.argtypes = [bp, C.c_double, dp, dp, C.c_int, dp]
        L.orc_daughter_elong.restype = C.c_int
        L.orc_daughter_elong.argtypes = [bp, dp, C.c_double, C.c_int, C.c_int, C.c_double,
                                         C.c_int, C.c_int, dp, dp, dp, dp]
        L.orc_daughters_elong.restype = C.c_int
        L.orc_daughters_elong.argtypes = [bp, C.c_int, dp, dp, dp, C.c_uint, C.c_int, C.c_int,
                                          C.c_int, dp, dp, C.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Bulk:
    """One bulk WCA system (Example 1).  Q = g T tau_T^2 with g = 3N (Eq. 5)."""
    n: int
    L: tuple
    dt: float = 0.0025
    T: float = 0.722
    tau_T: float = 0.25
    g: float | None = None
    rc: float = RC_WCA
    use_cells: bool = True

    @property
    def V(self) -> float:
        return float(self.L[0] * self.L[1] * self.L[2])

    @property
    def dof(self) -> float:
        return float(3 * self.n) if self.g is None else float(self.g)

    @property
    def Q(self) -> float:
        return self.dof * self.T * self.tau_T ** 2

    def c(self) -> _Bulk:
        b = _Bulk()
        b.n = self.n
        b.use_cells = 1 if self.use_cells else 0
        for d in range(3):
            b.L[d] = float(self.L[d])
        b.dt, b.T, b.Q, b.g, b.rc = self.dt, self.T, self.Q, self.dof, self.rc
        return b


def wca(r2: float):
    """(phi, f/r) of the WCA pair at squared distance r2 (Eq. 6)."""
    f = C.c_double()
    phi = lib().orc_wca(float(r2), C.byref(f))
    return phi, f.value


def forces(b: Bulk, state: np.ndarray, delta: float = 0.0, brute: bool | None = None):
    """F [3, N], virial W (xx yy zz xy xz yz) and U of state [6, N] (rows 0-2 used)."""
    n = b.n
    s = np.ascontiguousarray(state, dtype=np.float64)
    F = np.zeros((3, n))
    W = np.zeros(6)
    U = C.c_double()
    cb = b.c()
    if brute is not None:
        cb.use_cells = 0 if brute else 1
    rc = lib().orc_forces(C.byref(cb), float(delta), _p(s[0]), _p(s[1]), _p(s[2]),
                          _p(F[0]), _p(F[1]), _p(F[2]), _p(W), C.byref(U))
    if rc:
        raise RuntimeError("oracle forces failed")
    return F, W, U.value


def pressure(b: Bulk, state: np.ndarray, delta: float = 0.0):
    """(P[6] = xx yy zz xy xz yz, U, sum p^2) of a state [6, N]."""
    s = np.ascontiguousarray(state, dtype=np.float64)
    P = np.zeros(6)
    U, K2 = C.c_double(), C.c_double()
    if lib().orc_pressure(C.byref(b.c()), _p(s), float(delta), _p(P), C.byref(U), C.byref(K2)):
        raise RuntimeError("oracle pressure failed")
    return P, U.value, K2.value


def apply_mapping(b: Bulk, m: int, state: np.ndarray, alpha: float = 0.0,
                  reset_alpha: bool = False):
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.empty_like(s)
    a = C.c_double()
    lib().orc_apply_mapping(C.byref(b.c()), int(m), _p(s), float(alpha),
                            1 if reset_alpha else 0, _p(out), C.byref(a))
    return out, a.value


def trajectory(b: Bulk, state: np.ndarray, n_steps: int, gamma: float = 0.0,
               alpha: float = 0.0, delta: float = 0.0):
    """Run n_steps; returns (final state, alpha, delta, obs[n_steps+1, 8]) with
    obs columns K2, U, alpha, xi, Pxy, Wxy, delta, H_ext."""
    s = np.array(state, dtype=np.float64, order="C")
    a, d = C.c_double(alpha), C.c_double(delta)
    obs = np.zeros((n_steps + 1, 8))
    if lib().orc_trajectory(C.byref(b.c()), float(gamma), _p(s), C.byref(a), C.byref(d),
                            int(n_steps), _p(obs)):
        raise RuntimeError("oracle trajectory failed")
    return s, a.value, d.value, obs


def mother(b: Bulk, init: np.ndarray, n_eq: int, n_states: int, spacing: int,
           alpha0: float = 0.0):
    """Algorithm 2, mother part: states [n_states, 6, N] and alphas [n_states]."""
    s = np.ascontiguousarray(init, dtype=np.float64)
    out = np.zeros((n_states, 6, b.n))
    al = np.zeros(n_states)
    if lib().orc_mother(C.byref(b.c()), _p(s), float(alpha0), int(n_eq), int(n_states),
                        int(spacing), _p(out), _p(al)):
        raise RuntimeError("oracle mother failed")
    return out, al


def daughter(b: Bulk, mother_state: np.ndarray, mother_alpha: float, m: int, gamma: float,
             n_steps: int, sample_every: int = 1, reset_alpha: bool = False):
    """One daughter: (B[S], Omega, final state [6, N], final alpha)."""
    s = np.ascontiguousarray(mother_state, dtype=np.float64)
    S = n_steps // sample_every + 1
    B = np.zeros(S)
    om = C.c_double()
    fin = np.zeros((6, b.n))
    fa = C.c_double()
    if lib().orc_daughter(C.byref(b.c()), _p(s), float(mother_alpha), int(m),
                          1 if reset_alpha else 0, float(gamma), int(n_steps),
                          int(sample_every), _p(B), C.byref(om), _p(fin), C.byref(fa)):
        raise RuntimeError("oracle daughter failed")
    return B, om.value, fin, fa.value


def daughters(b: Bulk, mothers: np.ndarray, mother_alpha, gammas, n_steps: int,
              sample_every: int = 1, mapping_mask: int = 0xF, reset_alpha: bool = False,
              n_threads: int | None = None):
    """The ensemble: B [G*M, S] and Omega [G*M], daughter d = g*M + k for the
    k-th set bit m of mapping_mask (mapping codes 0..31, see apply_mapping)."""
    mothers = np.ascontiguousarray(mothers, dtype=np.float64)
    G = mothers.shape[0]
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(mother_alpha, np.float64), (G,)))
    gm = np.ascontiguousarray(np.broadcast_to(np.asarray(gammas, np.float64), (G,)))
    M = bin(mapping_mask & 0xFFFFFFFF).count("1")
    S = n_steps // sample_every + 1
    B = np.zeros((G * M, S))
    Om = np.zeros(G * M)
    nt = n_threads or os.cpu_count() or 1
    rc = lib().orc_daughters(C.byref(b.c()), G, _p(mothers), _p(al), _p(gm),
                             int(mapping_mask), 1 if reset_alpha else 0, int(n_steps),
                             int(sample_every), _p(B), _p(Om), int(nt))
    if rc:
        raise RuntimeError(f"oracle daughters failed ({rc})")
    return B, Om


# ------------------------------------------------- planar elongational flow --

def trajectory_elong(b: Bulk, state: np.ndarray, n_steps: int, eps: float,
                     alpha: float = 0.0):
    """Run n_steps under planar elongation grad u = diag(eps, 0, -eps) from
    the switch-on box b.L; returns (final state, alpha, obs[n_steps+1, 9])
    with obs columns K2, U, alpha, xi, Pxx-Pzz, Wxx-Wzz, Lx, Lz, H_ext."""
    s = np.array(state, dtype=np.float64, order="C")
    a = C.c_double(alpha)
    obs = np.zeros((n_steps + 1, 9))
    if lib().orc_trajectory_elong(C.byref(b.c()), float(eps), _p(s), C.byref(a),
                                  int(n_steps), _p(obs)):
        raise RuntimeError("oracle elongational trajectory failed")
    return s, a.value, obs


def daughter_elong(b: Bulk, mother_state: np.ndarray, mother_alpha: float, m: int,
                   eps: float, n_steps: int, sample_every: int = 1,
                   reset_alpha: bool = False):
    """One elongational daughter: (B[S] = P_xx - P_zz, Omega, final state, alpha)."""
    s = np.ascontiguousarray(mother_state, dtype=np.float64)
    S = n_steps // sample_every + 1
    B = np.zeros(S)
    om = C.c_double()
    fin = np.zeros((6, b.n))
    fa = C.c_double()
    if lib().orc_daughter_elong(C.byref(b.c()), _p(s), float(mother_alpha), int(m),
                                1 if reset_alpha else 0, float(eps), int(n_steps),
                                int(sample_every), _p(B), C.byref(om), _p(fin),
                                C.byref(fa)):
        raise RuntimeError("oracle elongational daughter failed")
    return B, om.value, fin, fa.value


def daughters_elong(b: Bulk, mothers: np.ndarray, mother_alpha, rates, n_steps: int,
                    sample_every: int = 1, mapping_mask: int = 0x30003,
                    reset_alpha: bool = False, n_threads: int | None = None):
    """The elongational ensemble, laid out as daughters(); the default set
    {identity, p -> -p, x <-> z, x <-> z with p -> -p} cancels Omega(0)."""
    mothers = np.ascontiguousarray(mothers, dtype=np.float64)
    G = mothers.shape[0]
    al = np.ascontiguousarray(np.broadcast_to(np.asarray(mother_alpha, np.float64), (G,)))
    er = np.ascontiguousarray(np.broadcast_to(np.asarray(rates, np.float64), (G,)))
    M = bin(mapping_mask & 0xFFFFFFFF).count("1")
    S = n_steps // sample_every + 1
    B = np.zeros((G * M, S))
    Om = np.zeros(G * M)
    nt = n_threads or os.cpu_count() or 1
    rc = lib().orc_daughters_elong(C.byref(b.c()), G, _p(mothers), _p(al), _p(er),
                                   int(mapping_mask), 1 if reset_alpha else 0,
                                   int(n_steps), int(sample_every), _p(B), _p(Om), int(nt))
    if rc:
        raise RuntimeError(f"oracle elongational daughters failed ({rc})")
    return B, Om
