"""ctypes binding of libidos.so: argument marshalling only.

Every call goes straight to the C ABI declared in include/idos.h; outputs are
numpy arrays allocated here and filled by the library.  CUDA streams are
passed as integer handles (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
MAX_LEVELS = 8
# Trailing update of the float32 two-stage reduction on the tensor cores with
# six split-bfloat16 products (float32-quality sums).
DEFAULT_TC_PRODUCTS = 6
GRAPHENE, TMDC = 0, 1
FP64, FP32_REFINE64 = 0, 1
SMOOTH_GAUSS, SMOOTH_POLY = 0, 1
_PRECISION = {"fp64": FP64, "fp32": FP32_REFINE64, FP64: FP64, FP32_REFINE64: FP32_REFINE64}
_SMOOTHING = {"gauss": SMOOTH_GAUSS, "poly": SMOOTH_POLY, SMOOTH_GAUSS: SMOOTH_GAUSS, SMOOTH_POLY: SMOOTH_POLY}
_KIND = {"graphene": GRAPHENE, "tmdc": TMDC, GRAPHENE: GRAPHENE, TMDC: TMDC}


class ModelDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("precision", C.c_int32), ("smoothing", C.c_int32), ("n_levels", C.c_int32),
        ("N", C.c_int32 * MAX_LEVELS), ("Kside", C.c_int32 * MAX_LEVELS),
        ("t", C.c_double), ("eps_onsite", C.c_double), ("a", C.c_double), ("p", C.c_double),
        ("sentinel", C.c_double), ("e_min", C.c_double), ("e_max", C.c_double), ("delta", C.c_double),
        ("n_E", C.c_int32), ("refine64_iters", C.c_int32), ("model_seed", C.c_uint64),
        ("workspace_bytes", C.c_int64), ("tc_products", C.c_int32), ("sm_split", C.c_int32), ("overlap_s", C.c_double),
        ("persistent", C.c_int32), ("graph", C.c_int32),
    ]


class MlmcOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("theta", C.c_double), ("c_alpha", C.c_double),
                ("pilot_samples", C.c_int64), ("work_model", C.c_int32), ("max_rounds", C.c_int32),
                ("seed", C.c_uint64)]


TUNE_MAX = 56


class Tuning(C.Structure):
    _fields_ = [("sm_split", C.c_int32), ("small_max_n", C.c_int32), ("best_ms", C.c_double),
                ("n_tried", C.c_int32), ("tried_split", C.c_int32 * TUNE_MAX), ("tried_small", C.c_int32 * TUNE_MAX),
                ("tried_ms", C.c_double * TUNE_MAX), ("persistent", C.c_int32),
                ("tried_persistent", C.c_int32 * TUNE_MAX), ("graph", C.c_int32),
                ("tried_graph", C.c_int32 * TUNE_MAX), ("w_tile", C.c_int32), ("chase_pair", C.c_int32),
                ("tried_w_tile", C.c_int32 * TUNE_MAX), ("tried_chase_pair", C.c_int32 * TUNE_MAX),
                ("placement", C.c_int32), ("tried_placement", C.c_int32 * TUNE_MAX),
                ("panel_cluster", C.c_int32), ("tried_panel_cluster", C.c_int32 * TUNE_MAX),
                ("her2k_lower", C.c_int32), ("tried_her2k_lower", C.c_int32 * TUNE_MAX),
                ("persist_reserve", C.c_int32), ("tried_persist_reserve", C.c_int32 * TUNE_MAX)]


class Estimate(C.Structure):
    _fields_ = [("mean", C.POINTER(C.c_double)), ("var", C.POINTER(C.c_double)),
                ("M", C.POINTER(C.c_int64)), ("V", C.POINTER(C.c_double)), ("W", C.POINTER(C.c_double)),
                ("seconds", C.c_double), ("rounds", C.c_int32), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64)]


class Rates(C.Structure):
    _fields_ = [("W", C.c_double), ("S", C.c_double), ("D", C.c_double), ("C", C.c_double),
                ("W_se", C.c_double), ("S_se", C.c_double), ("D_se", C.c_double), ("C_se", C.c_double),
                ("n_W", C.c_int32), ("n_S", C.c_int32), ("n_D", C.c_int32), ("n_C", C.c_int32),
                ("work_mc", C.c_double), ("work_mlmc", C.c_double), ("work_fs", C.c_double),
                ("theta_mc", C.c_double)]


class TraceEntry(C.Structure):
    _fields_ = [("kid", C.c_int32), ("lane", C.c_int32), ("launches", C.c_int32), ("reserved", C.c_int32),
                ("t0_ms", C.c_double), ("t1_ms", C.c_double)]


class IdosError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {status_string(status)} ({status}): {detail}")
        self.status = status


_LIB = None
_SYMBOLS = {
    "idos_create_model": (C.c_int, [C.POINTER(ModelDesc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "idos_destroy_model": (None, [C.c_void_p]),
    "idos_status_string": (C.c_char_p, [C.c_int]),
    "idos_last_error": (C.c_char_p, []),
    "idos_sample_level": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_int64, C.c_void_p]),
    "idos_sample_level_detail": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_int64,
                                           C.c_void_p, C.c_void_p, C.c_void_p]),
    "idos_sample_levels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]),
    "idos_get_level_stats": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_double)]),
    "idos_reset_level_stats": (C.c_int, [C.c_void_p, C.c_int]),
    "idos_get_level_moments": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.c_void_p,
                                         C.POINTER(C.c_double)]),
    "idos_combine_level_stats": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "idos_fit_rates": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.POINTER(Rates)]),
    "idos_eval_idos": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_uint64, C.c_int, C.c_int64,
                                 C.c_void_p, C.c_void_p]),
    "idos_mlmc_estimate": (C.c_int, [C.c_void_p, C.POINTER(MlmcOpts), C.POINTER(Estimate)]),
    "idos_vacancy_masks": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_int64, C.c_int64,
                                     C.c_void_p]),
    "idos_hamiltonian": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "idos_eigvalsh": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "idos_tridiagonalize": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "idos_her2k": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "idos_stage1_w": (C.c_int, [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "idos_get_partition": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_char_p)]),
    "idos_get_graph_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_char_p)]),
    "idos_server_create": (C.c_int, [C.POINTER(ModelDesc), C.c_int, C.c_int64, C.POINTER(C.c_void_p)]),
    "idos_server_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_int64, C.POINTER(C.c_int64)]),
    "idos_server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                   C.POINTER(C.c_double)]),
    "idos_server_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]),
    "idos_server_destroy": (None, [C.c_void_p]),
    "idos_dos_from_idos": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p]),
    "idos_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(Tuning)]),
    "idos_measure_fma_peak": (C.c_int, [C.c_int, C.c_int64, C.c_void_p, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "idos_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "idos_profile_count": (C.c_int, []),
    "idos_get_profile": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64)]),
    "idos_reset_profile": (C.c_int, [C.c_void_p]),
    "idos_get_trace": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_int64)]),
    "idos_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(Tuning)]),
    "idos_eval_idos_noalloc": (C.c_int, [C.POINTER(ModelDesc), C.c_int, C.c_int, C.c_void_p, C.c_uint64, C.c_int,
                                         C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
}


def lib_path() -> str:
    return os.path.join(HERE, "libidos.so")


def load_library():
    """Load libidos.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(python -m paper_1611_09784_gb300.build)")
    lib = C.CDLL(path)
    for name, (res, args) in _SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def status_string(status: int) -> str:
    return load_library().idos_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != 0:
        detail = load_library().idos_last_error().decode(errors="replace")
        raise IdosError(status, where, detail)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_desc(cfg: dict) -> ModelDesc:
    """ModelDesc from a plain dict (keys as in the C struct; levels as [(N, K), ...])."""
    d = ModelDesc()
    d.kind = _KIND[cfg.get("kind", "graphene")]
    d.precision = _PRECISION[cfg.get("precision", "fp32")]
    d.smoothing = _SMOOTHING[cfg.get("smoothing", "gauss")]
    levels = cfg["levels"]
    d.n_levels = len(levels)
    for i, (N, K) in enumerate(levels):
        d.N[i] = int(N)
        d.Kside[i] = int(K)
    d.t = float(cfg.get("t", -2.7))
    d.eps_onsite = float(cfg.get("eps_onsite", 0.0))
    d.a = float(cfg.get("a", 2.46))
    d.p = float(cfg.get("p", 0.05))
    d.sentinel = float(cfg.get("sentinel", 1.0e3))
    d.e_min = float(cfg.get("e_min", -9.0))
    d.e_max = float(cfg.get("e_max", 9.0))
    d.delta = float(cfg.get("delta", 0.1))
    d.n_E = int(cfg.get("n_E", 201))
    d.refine64_iters = int(cfg.get("refine64_iters", 0))
    d.model_seed = int(cfg.get("model_seed", 0))
    d.workspace_bytes = int(cfg.get("workspace_bytes", 0))
    d.tc_products = int(cfg.get("tc_products", DEFAULT_TC_PRODUCTS))
    d.sm_split = int(cfg.get("sm_split", -1))
    d.overlap_s = float(cfg.get("s", 0.0))
    d.persistent = int(cfg.get("persistent", -1))
    d.graph = int(cfg.get("graph", -1))
    return d


class Model:
    """Owner of one idos_model handle."""

    def __init__(self, cfg: dict, stream: int | None = None):
        lib = load_library()
        self.cfg = dict(cfg)
        self.desc = make_desc(cfg)
        self.n_E = self.desc.n_E
        self.n_levels = self.desc.n_levels
        self.kind = self.desc.kind
        # orbitals and vacancy sites per unit cell (graphene: 2 and 2; TMDC-shaped: 11 and 1)
        self.orb_per_cell = 11 if self.kind == TMDC else 2
        self.vac_per_cell = 1 if self.kind == TMDC else 2
        h = C.c_void_p()
        _check(lib.idos_create_model(C.byref(self.desc), C.c_void_p(stream or 0), C.byref(h)),
               "idos_create_model")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().idos_destroy_model(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sample_level(self, level: int, n_samples: int, seed: int, first_sample: int = 0,
                     want_Y: bool = False):
        Y = np.empty((n_samples, self.n_E)) if want_Y else None
        _check(load_library().idos_sample_level(self._h, level, n_samples, seed, first_sample, _ptr(Y)),
               "idos_sample_level")
        return Y

    def sample_levels(self, n_samples, seed: int, first_samples=None):
        """All levels at once (concurrent streams); n_samples[l] per level."""
        ns = np.ascontiguousarray(n_samples, dtype=np.int64)
        fs = None if first_samples is None else np.ascontiguousarray(first_samples, dtype=np.int64)
        _check(load_library().idos_sample_levels(self._h, _ptr(ns), seed, _ptr(fs)), "idos_sample_levels")

    def sample_level_detail(self, level: int, n_samples: int, seed: int, first_sample: int = 0):
        Y = np.empty((n_samples, self.n_E))
        Qf = np.empty((n_samples, self.n_E))
        Qc = np.empty((n_samples, 4, self.n_E)) if level > 0 else None
        _check(load_library().idos_sample_level_detail(self._h, level, n_samples, seed, first_sample,
                                                       _ptr(Y), _ptr(Qf), _ptr(Qc)),
               "idos_sample_level_detail")
        return Y, Qf, Qc

    def autotune(self, n_samples, reps: int = 1):
        """idos_autotune: time every candidate configuration on this allocation
        and install the fastest; returns the choice and the timings."""
        n = np.ascontiguousarray(list(n_samples) + [0] * (self.n_levels - len(n_samples)), dtype=np.int64)
        t = Tuning()
        _check(load_library().idos_autotune(self._h, _ptr(n), reps, C.byref(t)), "idos_autotune")
        tried = [{"sm_split": t.tried_split[i], "small_max_n": t.tried_small[i],
                  "persistent": t.tried_persistent[i], "graph": t.tried_graph[i], "w_tile": t.tried_w_tile[i],
                  "chase_pair": t.tried_chase_pair[i], "placement": t.tried_placement[i],
                  "panel_cluster": t.tried_panel_cluster[i], "her2k_lower": t.tried_her2k_lower[i],
                  "persist_reserve": t.tried_persist_reserve[i],
                  "ms": round(t.tried_ms[i], 3)} for i in range(t.n_tried)]
        return {"sm_split": t.sm_split, "small_max_n": t.small_max_n, "persistent": t.persistent,
                "graph": t.graph, "w_tile": t.w_tile, "chase_pair": t.chase_pair,
                "placement": t.placement, "panel_cluster": t.panel_cluster, "her2k_lower": t.her2k_lower,
                "persist_reserve": t.persist_reserve,
                "best_ms": round(t.best_ms, 3),
                "tried": tried}

    def set_tuning(self, tuning: dict):
        """idos_set_tuning: install a configuration (e.g. autotune()'s result;
        keys sm_split, small_max_n, persistent, graph, w_tile, chase_pair,
        placement, panel_cluster) without timing anything."""
        t = Tuning()
        for key in ("sm_split", "small_max_n", "persistent", "graph", "w_tile", "chase_pair", "placement",
                    "panel_cluster"):
            setattr(t, key, int(tuning[key]))
        t.her2k_lower = int(tuning.get("her2k_lower", 1))
        t.persist_reserve = int(tuning.get("persist_reserve", 0))
        _check(load_library().idos_set_tuning(self._h, C.byref(t)), "idos_set_tuning")

    def graph_info(self):
        """(calls that replayed a graph, captures made, reason graph mode was
        given up or "")."""
        r, c, why = C.c_int64(), C.c_int64(), C.c_char_p()
        _check(load_library().idos_get_graph_info(self._h, C.byref(r), C.byref(c), C.byref(why)),
               "idos_get_graph_info")
        return r.value, c.value, (why.value or b"").decode()

    def get_partition(self):
        """(SMs of the finest level, SMs of the others, reason when unsplit)."""
        a, b, why = C.c_int(0), C.c_int(0), C.c_char_p()
        _check(load_library().idos_get_partition(self._h, C.byref(a), C.byref(b), C.byref(why)), "idos_get_partition")
        return a.value, b.value, (why.value or b"").decode()

    def get_level_stats(self, level: int):
        s1 = np.empty(self.n_E)
        s2 = np.empty(self.n_E)
        M = C.c_int64()
        secs = C.c_double()
        _check(load_library().idos_get_level_stats(self._h, level, C.byref(M), _ptr(s1), _ptr(s2),
                                                   C.byref(secs)), "idos_get_level_stats")
        return int(M.value), s1, s2, float(secs.value)

    def get_level_moments(self, level: int):
        """(M, moments[4, n_E]: sum Y, sum Y^2, sum Q_l, sum Q_l^2, GPU seconds)."""
        mo = np.empty((4, self.n_E))
        M = C.c_int64()
        secs = C.c_double()
        _check(load_library().idos_get_level_moments(self._h, level, C.byref(M), _ptr(mo), C.byref(secs)),
               "idos_get_level_moments")
        return int(M.value), mo, float(secs.value)

    def reset_level_stats(self, level: int = -1):
        _check(load_library().idos_reset_level_stats(self._h, level), "idos_reset_level_stats")

    def eval_idos(self, N: int, K: int, mask=None, seed: int = 0, level: int = 0, sample: int = 0,
                  want_eigs: bool = False):
        Q = np.empty(self.n_E)
        E = np.empty((K * K, self.orb_per_cell * N * N)) if want_eigs else None
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        _check(load_library().idos_eval_idos(self._h, N, K, _ptr(m), seed, level, sample, _ptr(Q), _ptr(E)),
               "idos_eval_idos")
        return (Q, E) if want_eigs else Q

    def mlmc_estimate(self, tol: float, theta: float = 0.5, c_alpha: float = 1.96, pilot_samples: int = 16,
                      work_model: int = 0, max_rounds: int = 3, seed: int = 0):
        o = MlmcOpts(tol, theta, c_alpha, pilot_samples, work_model, max_rounds, seed)
        mean = np.empty(self.n_E)
        var = np.empty(self.n_E)
        M = np.empty(self.n_levels, dtype=np.int64)
        V = np.empty(self.n_levels)
        W = np.empty(self.n_levels)
        est = Estimate(mean.ctypes.data_as(C.POINTER(C.c_double)), var.ctypes.data_as(C.POINTER(C.c_double)),
                       M.ctypes.data_as(C.POINTER(C.c_int64)), V.ctypes.data_as(C.POINTER(C.c_double)),
                       W.ctypes.data_as(C.POINTER(C.c_double)), 0.0, 0, 0, 0)
        _check(load_library().idos_mlmc_estimate(self._h, C.byref(o), C.byref(est)), "idos_mlmc_estimate")
        return {"mean": mean, "var": var, "M": M, "V": V, "W": W, "seconds": est.seconds,
                "rounds": est.rounds, "h2d_bytes": est.h2d_bytes, "d2h_bytes": est.d2h_bytes}

    def set_profiling(self, enable=True):
        """True / 1: per-family totals, levels serialised on one stream;
        2: timeline (levels on their own streams and partition, trace kept);
        False / 0: off."""
        mode = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
        _check(load_library().idos_set_profiling(self._h, mode), "idos_set_profiling")

    def get_trace(self) -> list:
        """Timed scopes of the last timeline-mode idos_sample_levels call:
        [{"kernel", "lane", "launches", "t0_ms", "t1_ms"}] in issue order."""
        lib = load_library()
        n = C.c_int64()
        _check(lib.idos_get_trace(self._h, 0, None, C.byref(n)), "idos_get_trace")
        buf = (TraceEntry * max(1, n.value))()
        _check(lib.idos_get_trace(self._h, n.value, C.cast(buf, C.c_void_p), C.byref(n)), "idos_get_trace")
        out = []
        for e in buf[:n.value]:
            name = C.c_char_p()
            _check(lib.idos_get_profile(self._h, e.kid, C.byref(name), None, None), "idos_get_profile")
            out.append({"kernel": name.value.decode(), "lane": e.lane, "launches": e.launches,
                        "t0_ms": e.t0_ms, "t1_ms": e.t1_ms})
        return out

    def reset_profile(self):
        _check(load_library().idos_reset_profile(self._h), "idos_reset_profile")

    def get_profile(self) -> dict:
        """{kernel name: (total ms, launches)} for families that launched."""
        lib = load_library()
        out = {}
        for kid in range(lib.idos_profile_count()):
            name = C.c_char_p()
            ms = C.c_double()
            n = C.c_int64()
            _check(lib.idos_get_profile(self._h, kid, C.byref(name), C.byref(ms), C.byref(n)),
                   "idos_get_profile")
            if n.value:
                out[name.value.decode()] = (float(ms.value), int(n.value))
        return out

    def vacancy_masks(self, N: int, level: int, seed: int, first_sample: int, n_samples: int):
        out = np.empty((n_samples, self.vac_per_cell * N * N), dtype=np.uint8)
        _check(load_library().idos_vacancy_masks(self._h, N, level, seed, first_sample, n_samples, _ptr(out)),
               "idos_vacancy_masks")
        return out

    def hamiltonian(self, N: int, K: int, k_index: int, mask):
        n = self.orb_per_cell * N * N
        out = np.empty((n, n), dtype=np.complex128)
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        _check(load_library().idos_hamiltonian(self._h, N, K, k_index, _ptr(m), _ptr(out)), "idos_hamiltonian")
        return out


class Server:
    """Request loop over the level sampler (idos_server_*): submit() queues a
    request and returns a ticket, wait() returns (sum Y, sum Y^2, latency in
    seconds, device milliseconds) of its samples."""

    def __init__(self, cfg: dict, n_workers: int = 4, hbm_budget_bytes: int = 0):
        self.desc = make_desc(cfg)
        self.n_E = self.desc.n_E
        h = C.c_void_p()
        _check(load_library().idos_server_create(C.byref(self.desc), n_workers, hbm_budget_bytes, C.byref(h)),
               "idos_server_create")
        self._h = h

    def submit(self, level: int, n_samples: int, seed: int, first_sample: int = 0) -> int:
        t = C.c_int64(0)
        _check(load_library().idos_server_submit(self._h, level, n_samples, seed, first_sample, C.byref(t)),
               "idos_server_submit")
        return t.value

    def wait(self, ticket: int):
        s1 = np.empty(self.n_E)
        s2 = np.empty(self.n_E)
        lat, dev = C.c_double(0), C.c_double(0)
        _check(load_library().idos_server_wait(self._h, ticket, _ptr(s1), _ptr(s2), C.byref(lat), C.byref(dev)),
               "idos_server_wait")
        return s1, s2, lat.value, dev.value

    def info(self):
        vals = [C.c_int64(0) for _ in range(4)]
        _check(load_library().idos_server_info(self._h, *[C.byref(v) for v in vals]), "idos_server_info")
        return dict(zip(("completed", "queued", "in_flight_bytes", "peak_bytes"), (v.value for v in vals)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().idos_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dos_from_idos(Q, e_min: float, e_max: float):
    """Density of states from an IDoS on the uniform grid (idos_dos_from_idos)."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.empty_like(Q)
    _check(load_library().idos_dos_from_idos(_ptr(Q), Q.shape[-1], e_min, e_max, _ptr(out)), "idos_dos_from_idos")
    return out


def combine_level_stats(counts, sums):
    """Eq. (2.6) estimate and its variance (idos_combine_level_stats) from
    per-level sample counts (int64[L]) and sums (float64[L, 2, n_E]: sum Y,
    sum Y^2); levels with count 0 are left out."""
    M = np.ascontiguousarray(counts, dtype=np.int64)
    S = np.ascontiguousarray(sums, dtype=np.float64)
    if S.ndim != 3 or S.shape[0] != M.shape[0] or S.shape[1] != 2:
        raise ValueError("sums must have shape (levels, 2, n_E)")
    n_E = S.shape[2]
    mean = np.empty(n_E)
    var = np.empty(n_E)
    _check(load_library().idos_combine_level_stats(M.shape[0], _ptr(M), _ptr(S), n_E, _ptr(mean), _ptr(var)),
           "idos_combine_level_stats")
    return mean, var


def fit_rates(Ns, counts, moments, cost=None) -> dict:
    """Rates W, S, D, C of the complexity models and the work exponents they
    imply (idos_fit_rates).  Ns: supercell sides; counts: int64[L];
    moments: float64[L, 4, n_E] as Model.get_level_moments; cost: per-sample
    work per level or None."""
    N = np.ascontiguousarray(Ns, dtype=np.int32)
    M = np.ascontiguousarray(counts, dtype=np.int64)
    mo = np.ascontiguousarray(moments, dtype=np.float64)
    if mo.ndim != 3 or mo.shape[:2] != (M.shape[0], 4) or N.shape[0] != M.shape[0]:
        raise ValueError("moments must have shape (levels, 4, n_E)")
    c = None if cost is None else np.ascontiguousarray(cost, dtype=np.float64)
    r = Rates()
    _check(load_library().idos_fit_rates(M.shape[0], _ptr(N), _ptr(M), _ptr(mo), _ptr(c), mo.shape[2], C.byref(r)),
           "idos_fit_rates")
    return {name: getattr(r, name) for name, _ in Rates._fields_}


def measure_fma_peak(precision="fp32", iters: int = 1 << 16, stream: int | None = None):
    """(flop/s, ms) of the FMA microbenchmark (idos_measure_fma_peak)."""
    f, ms = C.c_double(0), C.c_double(0)
    _check(load_library().idos_measure_fma_peak(_PRECISION[precision], iters, C.c_void_p(stream or 0), C.byref(f),
                                                C.byref(ms)), "idos_measure_fma_peak")
    return f.value, ms.value


def create_model(cfg: dict, stream: int | None = None) -> Model:
    return Model(cfg, stream)


def eigvalsh(H, precision="fp32", refine64_iters: int = 0, stream: int | None = None,
             tc_products: int | None = None):
    """Eigenvalues of a batch of Hermitian matrices through the GPU path."""
    H = np.ascontiguousarray(H, dtype=np.complex128)
    if H.ndim == 2:
        H = H[None]
    batch, n, _ = H.shape
    out = np.empty((batch, n))
    tc = DEFAULT_TC_PRODUCTS if tc_products is None else int(tc_products)
    _check(load_library().idos_eigvalsh(_PRECISION[precision], refine64_iters, tc, n, batch, _ptr(H), _ptr(out),
                                        C.c_void_p(stream or 0)), "idos_eigvalsh")
    return out


def tridiagonalize(H, precision="fp32", stream: int | None = None, tc_products: int | None = None):
    """(d, e^2) of the hot path's reduction of a batch of Hermitian matrices
    (idos_tridiagonalize); e^2[:, i] couples rows i and i + 1."""
    H = np.ascontiguousarray(H, dtype=np.complex128)
    if H.ndim == 2:
        H = H[None]
    batch, n, _ = H.shape
    d = np.empty((batch, n))
    e2 = np.empty((batch, n))
    tc = DEFAULT_TC_PRODUCTS if tc_products is None else int(tc_products)
    _check(load_library().idos_tridiagonalize(_PRECISION[precision], tc, n, batch, _ptr(H), _ptr(d), _ptr(e2),
                                              C.c_void_p(stream or 0)), "idos_tridiagonalize")
    return d, e2


def stage1_w(A, YT, k: int = 0, mode: int = 2):
    """W = A22 (Y T) of one stage-1 panel through the large path's W kernel
    (float32 storage; mode 2 = tensor cores, 1 / 0 = FP32 pipe tiles).
    A: (batch, n, n) complex; YT: (batch, 16, n) complex; A22 = A[k+16:, k+16:]
    and V = YT[:, :, :m]; returns (batch, 16, n), entries m.. zero."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    YT = np.ascontiguousarray(YT, dtype=np.complex128)
    batch, n, _ = A.shape
    if YT.shape != (batch, 16, n):
        raise ValueError("YT must have shape (batch, 16, n)")
    out = np.empty_like(YT)
    _check(load_library().idos_stage1_w(int(mode), n, batch, int(k), _ptr(A), _ptr(YT), _ptr(out)), "idos_stage1_w")
    return out


def her2k(A, Y, Z, tc_products: int = DEFAULT_TC_PRODUCTS):
    """A - (Y Z^H + Z Y^H) through the large path's trailing-update kernel
    (float32 storage; tc_products 0 = FP32 pipe, 3 or 6 = tensor cores).
    A: (batch, n, n) complex; Y, Z: (batch, 16, n) complex (panel columns)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    Z = np.ascontiguousarray(Z, dtype=np.complex128)
    batch, n, _ = A.shape
    if Y.shape != (batch, 16, n) or Z.shape != (batch, 16, n):
        raise ValueError("Y and Z must have shape (batch, 16, n)")
    out = np.empty_like(A)
    _check(load_library().idos_her2k(int(tc_products), n, batch, _ptr(A), _ptr(Y), _ptr(Z), _ptr(out)), "idos_her2k")
    return out


def eval_idos_noalloc(cfg: dict, N: int, K: int, idos_dev_ptr: int, eigs_dev_ptr: int | None = None,
                      mask_dev_ptr: int | None = None, seed: int = 0, level: int = 0, sample: int = 0,
                      stream: int | None = None):
    """Allocation-free single-configuration IDoS (no model): inputs and outputs
    are caller-owned DEVICE pointers (integers, e.g. tensor.data_ptr()); the
    call enqueues on `stream` and returns without synchronising."""
    d = make_desc(cfg)
    _check(load_library().idos_eval_idos_noalloc(C.byref(d), N, K, C.c_void_p(mask_dev_ptr or 0), seed, level,
                                                 sample, C.c_void_p(idos_dev_ptr), C.c_void_p(eigs_dev_ptr or 0),
                                                 C.c_void_p(stream or 0)), "idos_eval_idos_noalloc")
