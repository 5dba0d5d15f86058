"""Thin ctypes binding of ``libttcf.so`` with the names of ``include/ttcf.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host arrays are numpy float64; device arrays may be torch CUDA
tensors.  PyTorch supplies device memory (its caching allocator, through the
``dev_alloc``/``dev_free`` hooks) and the stream.  There is no CPU fallback:
if the library or a GPU is missing, the call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TTCF_OK, TTCF_E_INVALID, TTCF_E_CUDA, TTCF_E_OOM, TTCF_E_NUMERIC, TTCF_E_TIMEOUT, TTCF_E_STATE = range(7)
TTCF_BULK_WCA, TTCF_CONFINED_LJ, TTCF_BULK_WCA_ELONG = 0, 1, 2
CONF_NSLAB = 40
CONF_NOBS = 2 + 2 * CONF_NSLAB + 2   # + the inner wall layers' p_x sums
TTCF_FP64, TTCF_MIXED = 0, 1
D_OK, D_NONFINITE, D_NBR_OVERFLOW, D_FAST_ATOM, D_ABORTED, D_ESCAPED = 0, 1, 2, 4, 8, 16

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# The C ABI exported by libttcf.so (kept in sync with include/ttcf.h).
EXPORTS = ("ttcf_config_default", "ttcf_create", "ttcf_spawn_daughters", "ttcf_run",
           "ttcf_response", "ttcf_viscosity", "ttcf_omega_mean", "ttcf_daughter_series", "ttcf_group_status",
           "ttcf_get_state", "ttcf_get_stats", "ttcf_sample_mothers", "ttcf_mother_acf",
           "ttcf_kick_states",
           "ttcf_forces", "ttcf_autotune",
           "ttcf_run_noalloc", "ttcf_cv_config_default", "ttcf_cv_data", "ttcf_cv_train",
           "ttcf_cv_apply", "ttcf_cv_get_model", "ttcf_cv_forward", "ttcf_cv_gradient",
           "ttcf_confined_params_default", "ttcf_spawn_confined", "ttcf_sample_mothers_confined",
           "ttcf_response_obs", "ttcf_friction", "ttcf_friction_equilibrium", "ttcf_save", "ttcf_load", "ttcf_destroy",
           "ttcf_last_error",
           "ttcf_version")


class Config(C.Structure):
    _fields_ = [("system", C.c_int), ("precision", C.c_int), ("dt", C.c_double),
                ("T", C.c_double), ("tau_T", C.c_double), ("dof_mode", C.c_int),
                ("n_steps", C.c_int), ("sample_every", C.c_int), ("mapping_mask", C.c_uint),
                ("reset_alpha", C.c_int), ("keep_state", C.c_int), ("skin", C.c_double),
                ("block_threads", C.c_int), ("kernel_variant", C.c_int), ("use_graph", C.c_int), ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN),
                ("dev_free", FREE_FN), ("alloc_user", C.c_void_p), ("timeout_s", C.c_double),
                ("cell_frac", C.c_double)]


class ConfinedParams(C.Structure):
    _fields_ = [("k", C.c_double), ("rc", C.c_double), ("c_ff", C.c_double), ("c_wf", C.c_double),
                ("c_ww", C.c_double), ("h", C.c_double), ("ww_on", C.c_int), ("pad_", C.c_int)]


class CvConfig(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("holdout", C.c_float),
                ("seed", C.c_ulonglong)]


CV_NF, CV_NP = 32, 20865


class Stats(C.Structure):
    _fields_ = [("ms_run", C.c_double), ("ms_spawn", C.c_double), ("ms_reduce", C.c_double),
                ("pairs_interacting", C.c_double), ("rebuilds", C.c_double),
                ("atom_steps", C.c_double), ("launches", C.c_int), ("block_threads", C.c_int),
                ("skin", C.c_double)]


class TTCFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ttcf status {status}: {msg}")
        self.status = status


_lib = None
_dp = C.POINTER(C.c_double)


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libttcf.so (optionally building it first).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
    L = C.CDLL(path)
    vp, ip = C.c_void_p, C.POINTER(C.c_int)
    L.ttcf_config_default.argtypes = [C.POINTER(Config)]
    L.ttcf_config_default.restype = None
    L.ttcf_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    L.ttcf_spawn_daughters.argtypes = [vp, C.c_int, _dp, C.c_int, vp, vp, vp, C.c_int, ip]
    L.ttcf_run.argtypes = [vp, C.c_int]
    L.ttcf_response.argtypes = [vp, C.c_int, C.c_int] + [_dp] * 7 + [C.c_int, ip]
    L.ttcf_viscosity.argtypes = [vp, C.c_int] + [_dp] * 5 + [C.c_int, ip]
    L.ttcf_omega_mean.argtypes = [vp, C.c_int, _dp, _dp]
    L.ttcf_friction_equilibrium.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp,
                                            _dp, _dp]
    L.ttcf_daughter_series.argtypes = [vp, C.c_int, _dp, _dp, C.c_size_t]
    L.ttcf_group_status.argtypes = [vp, C.c_int, ip, C.c_int]
    L.ttcf_get_state.argtypes = [vp, C.c_int, C.c_int, _dp, _dp, _dp]
    L.ttcf_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.ttcf_sample_mothers.argtypes = [vp, C.c_int, _dp, C.c_int, _dp, C.c_int, C.c_int,
                                      C.c_int, _dp, _dp]
    L.ttcf_forces.argtypes = [vp, C.c_int, _dp, C.c_int, C.c_double, _dp, _dp, _dp, _dp]
    L.ttcf_autotune.argtypes = [vp, C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_int, ip, _dp, _dp, _dp]
    L.ttcf_run_noalloc.argtypes = [C.POINTER(Config), C.c_int, _dp, C.c_int, vp, vp, vp, vp, vp, vp]
    L.ttcf_run_noalloc.restype = C.c_int
    fp = C.POINTER(C.c_float)
    L.ttcf_cv_config_default.argtypes = [C.POINTER(CvConfig)]
    L.ttcf_cv_config_default.restype = None
    L.ttcf_cv_data.argtypes = [vp, C.c_int, fp, _dp, C.c_size_t]
    L.ttcf_cv_train.argtypes = [vp, C.c_int, C.POINTER(CvConfig), _dp, C.c_int]
    L.ttcf_cv_apply.argtypes = [vp, C.c_int, C.c_int, _dp, _dp, _dp]
    L.ttcf_cv_get_model.argtypes = [vp, fp, _dp, _dp, _dp]
    L.ttcf_cv_forward.argtypes = [vp, fp, C.c_int, fp, fp]
    L.ttcf_cv_gradient.argtypes = [vp, fp, C.c_int, fp, fp, fp, _dp]
    for name in ("ttcf_cv_data", "ttcf_cv_train", "ttcf_cv_apply", "ttcf_cv_get_model",
                 "ttcf_cv_forward", "ttcf_cv_gradient"):
        getattr(L, name).restype = C.c_int
    L.ttcf_confined_params_default.argtypes = [C.POINTER(ConfinedParams)]
    L.ttcf_confined_params_default.restype = None
    L.ttcf_spawn_confined.argtypes = [vp, C.c_int, _dp, vp, vp, C.POINTER(ConfinedParams), C.c_int,
                                      vp, vp, vp, C.c_int, ip]
    L.ttcf_sample_mothers_confined.argtypes = [vp, C.c_int, _dp, vp, vp, C.POINTER(ConfinedParams),
                                               C.c_int, _dp, C.c_int, C.c_int, C.c_int, _dp, _dp, ip]
    L.ttcf_response_obs.argtypes = [vp, C.c_int, C.c_int, C.c_int] + [_dp] * 7 + [C.c_int, ip]
    L.ttcf_mother_acf.argtypes = [vp, C.c_int, _dp, C.c_int, _dp, C.c_int, C.c_int, C.c_int,
                                  _dp, _dp, _dp, _dp]
    L.ttcf_mother_acf.restype = C.c_int
    L.ttcf_kick_states.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_double, C.c_ulonglong, C.c_int,
                                   vp, C.c_int]
    L.ttcf_kick_states.restype = C.c_int
    L.ttcf_friction.argtypes = [vp, C.c_int, C.c_int] + [_dp] * 5 + [C.c_int, ip]
    L.ttcf_friction.restype = C.c_int
    L.ttcf_save.argtypes = [vp, C.c_char_p]
    L.ttcf_load.argtypes = [vp, C.c_char_p]
    for f in ("ttcf_spawn_confined", "ttcf_sample_mothers_confined", "ttcf_response_obs",
              "ttcf_save", "ttcf_load"):
        getattr(L, f).restype = C.c_int
    L.ttcf_destroy.argtypes = [vp]
    L.ttcf_destroy.restype = None
    L.ttcf_last_error.argtypes = [vp]
    L.ttcf_last_error.restype = C.c_char_p
    L.ttcf_version.restype = C.c_char_p
    for name in ("ttcf_create", "ttcf_spawn_daughters", "ttcf_run", "ttcf_response",
                 "ttcf_viscosity", "ttcf_daughter_series", "ttcf_group_status",
                 "ttcf_get_state", "ttcf_get_stats", "ttcf_sample_mothers", "ttcf_forces",
                 "ttcf_autotune"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _box(box) -> np.ndarray:
    b = _f64(box).reshape(-1)
    if b.size != 3:
        raise ValueError("box must have 3 entries")
    return b


def config_default() -> Config:
    c = Config()
    load().ttcf_config_default(C.byref(c))
    return c


class _TorchAllocator:
    """dev_alloc/dev_free hooks backed by torch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream))
            except Exception:
                return None

        def _free(ptr, stream, user):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Context:
    """Owns one ``ttcf_ctx``.  Methods mirror the C ABI names."""

    def __init__(self, cfg: Config | None = None, use_torch_allocator: bool = True,
                 torch_stream: bool = True, **overrides):
        L = load()
        self._L = L
        self.cfg = cfg if cfg is not None else config_default()
        for k, v in overrides.items():
            setattr(self.cfg, k, v)
        self._alloc = None
        try:
            import torch
            if torch.cuda.is_available():
                if torch_stream and not self.cfg.stream:
                    self.cfg.stream = torch.cuda.current_stream().cuda_stream
                if use_torch_allocator:
                    self._alloc = _TorchAllocator()
                    self.cfg.dev_alloc = self._alloc.alloc
                    self.cfg.dev_free = self._alloc.free
        except ImportError:
            pass
        h = C.c_void_p()
        st = L.ttcf_create(C.byref(self.cfg), C.byref(h))
        if st != TTCF_OK:
            raise TTCFError(st, L.ttcf_last_error(None).decode())
        self.h = h

    # -- helpers --
    def _check(self, st: int, allowed=(TTCF_OK,)):
        if st not in allowed:
            raise TTCFError(st, self._L.ttcf_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self._L.ttcf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def n_samples(self) -> int:
        return self.cfg.n_steps // self.cfg.sample_every + 1

    @property
    def n_maps(self) -> int:
        return bin(self.cfg.mapping_mask & 0xFFFFFFFF).count("1")

    # -- C ABI --
    def spawn_daughters(self, mother_soa, mother_alpha=None, shear_rates=0.0, box=None) -> int:
        """mother_soa [G, 6, N] (numpy host or torch CUDA tensor)."""
        is_dev = hasattr(mother_soa, "is_cuda") and mother_soa.is_cuda
        if is_dev:
            import torch
            ms = mother_soa.contiguous().to(torch.float64)
            G, _, N = ms.shape
            al = None if mother_alpha is None else torch.as_tensor(
                mother_alpha, dtype=torch.float64, device=ms.device).expand(G).contiguous()
            gm = torch.as_tensor(shear_rates, dtype=torch.float64, device=ms.device).expand(G).contiguous()
            keep = (ms, al, gm)
            p_ms, p_al, p_gm = ms.data_ptr(), (al.data_ptr() if al is not None else None), gm.data_ptr()
        else:
            ms = _f64(mother_soa)
            G, _, N = ms.shape
            al = None if mother_alpha is None else _f64(np.broadcast_to(mother_alpha, (G,)))
            gm = _f64(np.broadcast_to(np.asarray(shear_rates, np.float64), (G,)))
            keep = (ms, al, gm)
            p_ms = ms.ctypes.data
            p_al = al.ctypes.data if al is not None else None
            p_gm = gm.ctypes.data
        if box is None:
            raise ValueError("box is required")
        bx = _box(box)
        bid = C.c_int(-1)
        self._check(self._L.ttcf_spawn_daughters(self.h, int(N), _ptr(bx), int(G), p_ms, p_al,
                                                 p_gm, 1 if is_dev else 0, C.byref(bid)))
        del keep
        return bid.value

    def run(self, n_steps: int = 0, allow_numeric: bool = False) -> int:
        allowed = (TTCF_OK, TTCF_E_NUMERIC) if allow_numeric else (TTCF_OK,)
        return self._check(self._L.ttcf_run(self.h, int(n_steps)), allowed)

    def response(self, batch: int, corrected: bool = False) -> dict:
        S = self.n_samples
        arr = {k: np.zeros(S) for k in ("t", "dav", "dav_se", "corr", "corr_se", "ttcf", "ttcf_se")}
        n = C.c_int()
        self._check(self._L.ttcf_response(self.h, batch, 1 if corrected else 0, _ptr(arr["t"]),
                                          _ptr(arr["dav"]), _ptr(arr["dav_se"]), _ptr(arr["corr"]),
                                          _ptr(arr["corr_se"]), _ptr(arr["ttcf"]),
                                          _ptr(arr["ttcf_se"]), S, C.byref(n)))
        return arr

    def viscosity(self, batch: int) -> dict:
        S = self.n_samples
        arr = {k: np.zeros(S) for k in ("t", "eta_ttcf", "eta_ttcf_se", "eta_dav", "eta_dav_se")}
        n = C.c_int()
        self._check(self._L.ttcf_viscosity(self.h, batch, _ptr(arr["t"]), _ptr(arr["eta_ttcf"]),
                                           _ptr(arr["eta_ttcf_se"]), _ptr(arr["eta_dav"]),
                                           _ptr(arr["eta_dav_se"]), S, C.byref(n)))
        return arr

    def omega_mean(self, batch: int):
        """(<Omega(0)> over the valid groups' daughters, number of valid groups)."""
        om, n = C.c_double(), C.c_double()
        self._check(self._L.ttcf_omega_mean(self.h, batch, C.byref(om), C.byref(n)))
        return om.value, int(n.value)

    def daughter_series(self, batch: int, n_daughters: int, n_obs: int = 1):
        """B [D, S] (n_obs = 1) or [D, n_obs, S], Omega [D]."""
        S = self.n_samples
        B = np.zeros((n_daughters, S) if n_obs == 1 else (n_daughters, n_obs, S))
        Om = np.zeros(n_daughters)
        self._check(self._L.ttcf_daughter_series(self.h, batch, _ptr(B), _ptr(Om), B.size))
        return B, Om

    def response_obs(self, batch: int, observable: int, corrected: bool = False) -> dict:
        S = self.n_samples
        arr = {k: np.zeros(S) for k in ("t", "dav", "dav_se", "corr", "corr_se", "ttcf", "ttcf_se")}
        n = C.c_int()
        self._check(self._L.ttcf_response_obs(self.h, batch, int(observable), 1 if corrected else 0,
                                              _ptr(arr["t"]), _ptr(arr["dav"]), _ptr(arr["dav_se"]),
                                              _ptr(arr["corr"]), _ptr(arr["corr_se"]),
                                              _ptr(arr["ttcf"]), _ptr(arr["ttcf_se"]), S, C.byref(n)))
        return arr

    def friction(self, batch: int, wall: int) -> dict:
        """Slip velocity and friction coefficient at wall 0 (bottom) or 1
        (top) of a confined batch (Eq. 12), TTCF and direct average."""
        S = self.n_samples
        arr = {k: np.zeros(S) for k in ("t", "slip_ttcf", "slip_dav", "xi_ttcf", "xi_dav")}
        n = C.c_int()
        self._check(self._L.ttcf_friction(self.h, batch, int(wall), _ptr(arr["t"]),
                                          _ptr(arr["slip_ttcf"]), _ptr(arr["slip_dav"]),
                                          _ptr(arr["xi_ttcf"]), _ptr(arr["xi_dav"]), S, C.byref(n)))
        return arr

    def friction_equilibrium(self, batch: int, wall: int, max_lag: int, s_grid) -> dict:
        """Equilibrium friction coefficient xi_0 (Eq. 12) of a zero-shear
        confined batch (see ttcf_friction_equilibrium)."""
        s = _f64(s_grid).reshape(-1)
        out = np.zeros(4)
        cf, cv = np.zeros(max_lag + 1), np.zeros(max_lag + 1)
        z = np.zeros(s.size)
        self._check(self._L.ttcf_friction_equilibrium(self.h, batch, int(wall), int(max_lag), int(s.size),
                                                      _ptr(s), _ptr(out), _ptr(cf), _ptr(cv), _ptr(z)))
        return {"xi0": out[0], "zeta0": out[1], "tau_m": out[2], "xi_ratio": out[3],
                "c_dvf": cf, "c_dvdv": cv, "zeta_s": z, "s": s}

    def save(self, path: str):
        self._check(self._L.ttcf_save(self.h, os.fsencode(path)))

    def load(self, path: str):
        self._check(self._L.ttcf_load(self.h, os.fsencode(path)))

    def spawn_confined(self, mother_soa, types, lattice, box, mother_alpha=None, shear_rates=0.0,
                       params: "ConfinedParams | None" = None) -> int:
        """Confined daughters (Example 2) from host arrays: mother_soa
        [G, 6, N], types [N] (0 fluid, 1 bottom, 2 top wall), lattice [3, N]."""
        ms = _f64(mother_soa)
        if ms.ndim == 2:
            ms = ms[None]
        G, _, N = ms.shape
        ty = np.ascontiguousarray(types, dtype=np.int32)
        lt = _f64(lattice)
        al = None if mother_alpha is None else _f64(np.broadcast_to(mother_alpha, (G,)))
        gm = _f64(np.broadcast_to(np.asarray(shear_rates, np.float64), (G,)))
        pr = params if params is not None else confined_params_default()
        bid = C.c_int(-1)
        self._check(self._L.ttcf_spawn_confined(self.h, int(N), _ptr(_box(box)), ty.ctypes.data,
                                                lt.ctypes.data, C.byref(pr), int(G), ms.ctypes.data,
                                                al.ctypes.data if al is not None else None,
                                                gm.ctypes.data, 0, C.byref(bid)))
        return bid.value

    def sample_mothers_confined(self, init_soa, types, lattice, box, n_eq: int, n_states: int,
                                spacing: int, params: "ConfinedParams | None" = None,
                                allow_numeric: bool = False):
        """(states [n_init, n_states, 6, N], alpha [n_init, n_states]); with
        allow_numeric also the per-chain status (flagged chains: TTCF_D_*)."""
        init = _f64(init_soa)
        if init.ndim == 2:
            init = init[None]
        n_init, _, N = init.shape
        ty = np.ascontiguousarray(types, dtype=np.int32)
        lt = _f64(lattice)
        out = np.zeros((n_init, n_states, 6, N))
        al = np.zeros((n_init, n_states))
        pr = params if params is not None else confined_params_default()
        cs = np.zeros(n_init, dtype=np.int32)
        allowed = (TTCF_OK, TTCF_E_NUMERIC) if allow_numeric else (TTCF_OK,)
        self._check(self._L.ttcf_sample_mothers_confined(
            self.h, int(N), _ptr(_box(box)), ty.ctypes.data, lt.ctypes.data, C.byref(pr),
            int(n_init), _ptr(init), int(n_eq), int(n_states), int(spacing), _ptr(out), _ptr(al),
            cs.ctypes.data_as(C.POINTER(C.c_int))), allowed)
        if allow_numeric:
            return out, al, cs
        return out, al

    def group_status(self, batch: int, n_groups: int) -> np.ndarray:
        st = np.zeros(n_groups, dtype=np.int32)
        self._check(self._L.ttcf_group_status(self.h, batch,
                                              st.ctypes.data_as(C.POINTER(C.c_int)), n_groups))
        return st

    def get_state(self, batch: int, daughter: int, n_atoms: int):
        soa = np.zeros((6, n_atoms))
        a, d = C.c_double(), C.c_double()
        self._check(self._L.ttcf_get_state(self.h, batch, daughter, _ptr(soa), C.byref(a), C.byref(d)))
        return soa, a.value, d.value

    def get_stats(self) -> dict:
        s = Stats()
        self._check(self._L.ttcf_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def sample_mothers(self, init_soa, box, n_eq: int, n_states: int, spacing: int):
        init = _f64(init_soa)
        if init.ndim == 2:
            init = init[None]
        n_init, _, N = init.shape
        out = np.zeros((n_init, n_states, 6, N))
        al = np.zeros((n_init, n_states))
        self._check(self._L.ttcf_sample_mothers(self.h, int(N), _ptr(_box(box)), int(n_init),
                                                _ptr(init), int(n_eq), int(n_states), int(spacing),
                                                _ptr(out), _ptr(al)))
        return out, al

    def mother_acf(self, init_soa, box, n_eq: int, n_steps: int, max_lag: int,
                   want_series: bool = False) -> dict:
        """Equilibrium P_xy correlations and the Green-Kubo integral along
        GPU mother trajectories (see ttcf_mother_acf)."""
        init = _f64(init_soa)
        if init.ndim == 2:
            init = init[None]
        n_init, _, N = init.shape
        out = {k: np.zeros(max_lag + 1) for k in ("acf_pxy", "acf_pxy2", "eta_gk")}
        ser = np.zeros((n_init, n_steps)) if want_series else None
        self._check(self._L.ttcf_mother_acf(self.h, int(N), _ptr(_box(box)), int(n_init), _ptr(init),
                                            int(n_eq), int(n_steps), int(max_lag),
                                            _ptr(out["acf_pxy"]), _ptr(out["acf_pxy2"]),
                                            _ptr(out["eta_gk"]),
                                            _ptr(ser) if ser is not None else None))
        if ser is not None:
            out["series"] = ser
        return out

    def kick_states(self, state_soa, n_copies: int, kick: float, seed: int, types=None,
                    keep_energy: bool = True):
        """n_copies copies [n, 6, N] of one phase point [6, N] with small random
        momentum kicks (see ttcf_kick_states): numpy in and out, or a torch
        CUDA tensor in and a torch CUDA tensor out."""
        is_dev = hasattr(state_soa, "is_cuda") and state_soa.is_cuda
        if is_dev:
            import torch
            st = state_soa.contiguous().to(torch.float64)
            N = st.shape[1]
            ty = None if types is None else torch.as_tensor(types, dtype=torch.int32, device=st.device).contiguous()
            out = torch.empty((n_copies, 6, N), dtype=torch.float64, device=st.device)
            p_st, p_ty, p_out = st.data_ptr(), (ty.data_ptr() if ty is not None else None), out.data_ptr()
            keep = (st, ty)
        else:
            st = _f64(state_soa)
            N = st.shape[1]
            ty = None if types is None else np.ascontiguousarray(types, dtype=np.int32)
            out = np.zeros((n_copies, 6, N))
            p_st, p_ty, p_out = st.ctypes.data, (ty.ctypes.data if ty is not None else None), out.ctypes.data
            keep = (st, ty)
        self._check(self._L.ttcf_kick_states(self.h, int(N), p_st, p_ty, int(n_copies), float(kick),
                                             int(seed) & 0xFFFFFFFFFFFFFFFF, 1 if keep_energy else 0, p_out,
                                             1 if is_dev else 0))
        del keep
        return out

    def autotune(self, soa, box, shear_rate: float = 1e-3, n_steps: int = 100):
        """Pick the fastest launch variant, skin and list-cell width for this
        N (cached in the context for later spawns); returns (variant, skin,
        cell_frac, ms)."""
        s = _f64(soa)
        if s.ndim == 2:
            s = s[None]
        n, _, N = s.shape
        v, sk, fr, ms = C.c_int(), C.c_double(), C.c_double(), C.c_double()
        self._check(self._L.ttcf_autotune(self.h, int(N), _ptr(_box(box)), int(n), _ptr(s),
                                          float(shear_rate), int(n_steps), C.byref(v),
                                          C.byref(sk), C.byref(fr), C.byref(ms)))
        return v.value, sk.value, fr.value, ms.value

    # -- learned control variate --
    def cv_data(self, batch: int, n_daughters: int):
        X = np.zeros((n_daughters, CV_NF), dtype=np.float32)
        z = np.zeros(n_daughters)
        self._check(self._L.ttcf_cv_data(self.h, batch, _fptr(X), _ptr(z), n_daughters))
        return X, z

    def cv_train(self, batch: int, cfg: CvConfig | None = None) -> np.ndarray:
        cfg = cfg or cv_config_default()
        loss = np.zeros(cfg.epochs)
        self._check(self._L.ttcf_cv_train(self.h, batch, C.byref(cfg), _ptr(loss), cfg.epochs))
        return loss

    def cv_apply(self, batch: int, aux_soa, aux_alpha=None) -> dict:
        """aux_soa [n, 6, N]: numpy host array or torch CUDA tensor (aux_alpha
        of the same kind, or None)."""
        out = np.zeros(8)
        if hasattr(aux_soa, "is_cuda") and aux_soa.is_cuda:
            import torch
            a = aux_soa.contiguous().to(torch.float64)
            al = None if aux_alpha is None else torch.as_tensor(aux_alpha, dtype=torch.float64,
                                                                device=a.device).contiguous()
            pa, pal = C.cast(a.data_ptr(), _dp), (C.cast(al.data_ptr(), _dp) if al is not None else None)
        else:
            a = _f64(aux_soa)
            al = None if aux_alpha is None else _f64(aux_alpha)
            pa, pal = _ptr(a), (None if al is None else _ptr(al))
        self._check(self._L.ttcf_cv_apply(self.h, batch, int(a.shape[0]), pa, pal, _ptr(out)))
        keys = ("eta_plain", "se_plain", "eta_cv", "se_cv", "c", "gain", "n_groups", "n_aux")
        return dict(zip(keys, out.tolist()))

    def cv_get_model(self):
        p = np.zeros(CV_NP, dtype=np.float32)
        fs = np.zeros((CV_NF, 2))
        zs = np.zeros(2)
        c = C.c_double()
        self._check(self._L.ttcf_cv_get_model(self.h, _fptr(p), _ptr(fs), _ptr(zs), C.byref(c)))
        return p, fs, zs, c.value

    def cv_forward(self, params, X):
        p = np.ascontiguousarray(params, dtype=np.float32)
        Xf = np.ascontiguousarray(X, dtype=np.float32)
        out = np.zeros(Xf.shape[0], dtype=np.float32)
        self._check(self._L.ttcf_cv_forward(self.h, _fptr(p), int(Xf.shape[0]), _fptr(Xf), _fptr(out)))
        return out

    def cv_gradient(self, params, X, y):
        p = np.ascontiguousarray(params, dtype=np.float32)
        Xf = np.ascontiguousarray(X, dtype=np.float32)
        yf = np.ascontiguousarray(y, dtype=np.float32)
        g = np.zeros(CV_NP, dtype=np.float32)
        loss = C.c_double()
        self._check(self._L.ttcf_cv_gradient(self.h, _fptr(p), int(Xf.shape[0]), _fptr(Xf), _fptr(yf),
                                             _fptr(g), C.byref(loss)))
        return g, loss.value

    def forces(self, soa, box, delta: float = 0.0):
        s = _f64(soa)
        if s.ndim == 2:
            s = s[None]
        n, _, N = s.shape
        F = np.zeros((n, 3, N))
        W = np.zeros((n, 6))
        U = np.zeros(n)
        self._check(self._L.ttcf_forces(self.h, int(N), _ptr(_box(box)), int(n), float(delta),
                                        _ptr(s), _ptr(F), _ptr(W), _ptr(U)))
        return F, W, U


def confined_params_default() -> ConfinedParams:
    p = ConfinedParams()
    load().ttcf_confined_params_default(C.byref(p))
    return p


def cv_config_default() -> CvConfig:
    c = CvConfig()
    load().ttcf_cv_config_default(C.byref(c))
    return c


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_float))


def run_noalloc(cfg: Config, mother_soa, mother_alpha, shear_rates, box, B, Omega, status) -> int:
    """ttcf_run_noalloc: every array is a torch CUDA tensor owned by the
    caller (float64 mothers [G,6,N], alpha [G] or None, rates [G]; outputs
    B [D,S] float64, Omega [D] float64, status [D] int32).  Enqueues on
    cfg.stream and returns the status code."""
    import torch
    L = load()
    bx = _box(box)

    def need(name, t, dtype, shape):
        if t is None or not t.is_cuda or not t.is_contiguous() or t.dtype != dtype or tuple(t.shape) != shape:
            raise ValueError(f"run_noalloc: {name} must be a contiguous CUDA {dtype} tensor of shape {shape}")

    if mother_soa is None or mother_soa.dim() != 3 or mother_soa.shape[1] != 6:
        raise ValueError("run_noalloc: mother_soa must have shape [G, 6, N]")
    G, _, N = mother_soa.shape
    D = G * bin(cfg.mapping_mask & 0xF).count("1")
    S = cfg.n_steps // max(cfg.sample_every, 1) + 1
    need("mother_soa", mother_soa, torch.float64, (G, 6, N))
    if mother_alpha is not None:
        need("mother_alpha", mother_alpha, torch.float64, (G,))
    need("shear_rates", shear_rates, torch.float64, (G,))
    need("B", B, torch.float64, (D, S))
    need("Omega", Omega, torch.float64, (D,))
    need("status", status, torch.int32, (D,))
    return L.ttcf_run_noalloc(C.byref(cfg), int(N), _ptr(bx), int(G), mother_soa.data_ptr(),
                              None if mother_alpha is None else mother_alpha.data_ptr(),
                              shear_rates.data_ptr(), B.data_ptr(), Omega.data_ptr(),
                              status.data_ptr())


def last_error() -> str:
    return load().ttcf_last_error(None).decode()


def version() -> str:
    return load().ttcf_version().decode()
