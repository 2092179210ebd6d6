"""Python binding of the GB300 lattice Abelian-Higgs library (libah.so).

Thin ctypes marshalling over the C ABI of include/ah.h, with the same names
(``ah_create``, ``ah_step``, ``ah_observables`` ...).  Every step of the
method runs in the library's CUDA kernels; there is no Python or CPU
fallback: importing works anywhere, but the first call that needs the library
raises if libah.so is missing or no CUDA device is present.

``Sim`` wraps a handle for convenience (context manager, numpy field access).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

AH_OK, AH_ERR_ARG, AH_ERR_OOM, AH_ERR_CUDA, AH_ERR_UNSTABLE = 0, 1, 2, 3, 4
AH_ERR_NONFINITE, AH_ERR_TIMEOUT, AH_ERR_BUSY, AH_ERR_CANCELLED, AH_ERR_NOTFOUND = 5, 6, 7, 8, 9
AH_MINKOWSKI, AH_RADIATION, AH_MATTER = 0, 1, 2
AH_FP32, AH_FP64 = 0, 1
AH_KERNEL_AUTO, AH_KERNEL_PLAIN, AH_KERNEL_FUSED = 0, 1, 2
AH_FLAG_EXACT_DIAG, AH_FLAG_AUTOTUNE, AH_FLAG_WRAP_THETA, AH_FLAG_CORE_GROWTH, AH_FLAG_TWO_STEP = 1, 2, 4, 8, 16
AH_FLAG_FUSED_DIAG = 32
AH_BATCH_AUTOTUNE, AH_BATCH_NO_GRAPH, AH_BATCH_TWO_STEP = 1, 2, 4

SUM_NAMES = ("L", "rho", "p", "K", "G2", "V", "Eel", "B", "KV", "G2V", "KL", "G2L", "pL", "rhoL",
             "gauss2", "gscale2")


class AhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("ah status %d: %s" % (status, msg))
        self.status = status


class ah_config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("era", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("s", ctypes.c_double), ("lambda0", ctypes.c_double), ("e0", ctypes.c_double),
                ("sigma", ctypes.c_double), ("tau0", ctypes.c_double), ("tau_end", ctypes.c_double),
                ("tau_ref", ctypes.c_double), ("seed", ctypes.c_uint64), ("diag_every", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class ah_obs(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("a", ctypes.c_double), ("step", ctypes.c_int64),
                ("n_sites", ctypes.c_int64), ("L_mean", ctypes.c_double), ("xi_L", ctypes.c_double),
                ("xi_W", ctypes.c_double), ("n_pierced", ctypes.c_int64), ("sum_abs_W", ctypes.c_int64),
                ("R_V", ctypes.c_double), ("R_L", ctypes.c_double), ("v2_V", ctypes.c_double),
                ("v2_L", ctypes.c_double), ("p_over_rho_L", ctypes.c_double), ("v2_omega", ctypes.c_double),
                ("gauss_rms", ctypes.c_double), ("gauss_max", ctypes.c_double), ("gauss_rel", ctypes.c_double),
                ("energy", ctypes.c_double), ("max_abs_theta", ctypes.c_double),
                ("sums", ctypes.c_double * 16), ("wind_abs_plane", ctypes.c_int64 * 3),
                ("wind_plane", ctypes.c_int64 * 3), ("nonfinite", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        d["sum"] = dict(zip(SUM_NAMES, d["sums"]))
        return d


class ah_batch_stats(ctypes.Structure):
    _fields_ = [("seconds", ctypes.c_double), ("setup_seconds", ctypes.c_double), ("site_updates", ctypes.c_double),
                ("sims_per_hour", ctypes.c_double), ("shape", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("weak_field_launches", ctypes.c_int64)]


class ah_window(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int32), ("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("z0", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("out", ctypes.c_void_p)]


class ah_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("running", ctypes.c_int32), ("queued", ctypes.c_int32), ("hbm_used", ctypes.c_int64),
                ("site_updates", ctypes.c_double), ("launches", ctypes.c_int64)]


class ah_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("n_sites", ctypes.c_int64), ("precision", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("state_bytes", ctypes.c_int64), ("step_bytes", ctypes.c_int64),
                ("step_launches", ctypes.c_int64), ("variant", ctypes.c_int32), ("n_variants", ctypes.c_int32),
                ("variant_name", ctypes.c_char * 32), ("fused_diag_passes", ctypes.c_int64),
                ("weak_field_launches", ctypes.c_int64)]


_SIGS = {
    "ah_abi_version": ([], ctypes.c_int),
    "ah_last_error": ([], ctypes.c_char_p),
    "ah_config_default": ([ctypes.POINTER(ah_config), ctypes.c_int32], None),
    "ah_create": ([ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                   ctypes.c_double, ctypes.c_double, ctypes.c_uint64], ctypes.c_void_p),
    "ah_create_ex": ([ctypes.POINTER(ah_config), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "ah_step": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "ah_observables": ([ctypes.c_void_p, ctypes.POINTER(ah_obs)], ctypes.c_int),
    "ah_observables_start": ([ctypes.c_void_p], ctypes.c_int),
    "ah_observables_finish": ([ctypes.c_void_p, ctypes.POINTER(ah_obs)], ctypes.c_int),
    "ah_observables_box": ([ctypes.c_void_p] + [ctypes.c_int32] * 6 + [ctypes.POINTER(ah_obs)], ctypes.c_int),
    "ah_get_fields": ([ctypes.c_void_p] + [ctypes.c_int32] * 6 + [ctypes.c_void_p], ctypes.c_int),
    "ah_set_fields": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "ah_set_stream": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ah_sync": ([ctypes.c_void_p], ctypes.c_int),
    "ah_get_step": ([ctypes.c_void_p], ctypes.c_int64),
    "ah_get_tau": ([ctypes.c_void_p], ctypes.c_double),
    "ah_get_info": ([ctypes.c_void_p, ctypes.POINTER(ah_info)], ctypes.c_int),
    "ah_destroy": ([ctypes.c_void_p], None),
    "ah_variant_count": ([ctypes.c_int32], ctypes.c_int32),
    "ah_set_variant": ([ctypes.c_void_p, ctypes.c_int32], ctypes.c_int),
    "ah_autotune": ([ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "ah_observables_noalloc": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.POINTER(ah_config),
                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "ah_batch_run": ([ctypes.POINTER(ah_config), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ah_obs),
                      ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ah_batch_stats)], ctypes.c_int),
    "ah_batch_run_ex": ([ctypes.POINTER(ah_config), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ah_obs),
                         ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ah_batch_stats),
                         ctypes.POINTER(ah_window), ctypes.c_int32], ctypes.c_int),
    "ah_server_submit_ex": ([ctypes.c_void_p, ctypes.POINTER(ah_config), ctypes.POINTER(ah_window), ctypes.c_int32,
                             ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "ah_server_create": ([ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
                         ctypes.c_int),
    "ah_server_submit": ([ctypes.c_void_p, ctypes.POINTER(ah_config), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "ah_server_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ah_obs), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "ah_server_cancel": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "ah_server_stats_get": ([ctypes.c_void_p, ctypes.POINTER(ah_server_stats)], ctypes.c_int),
    "ah_server_destroy": ([ctypes.c_void_p], None),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libah.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libah.so not built (%s); run paper_1809_00995_gb300._build.build()"
                                   % _build.LIB)
            lib = ctypes.CDLL(_build.LIB)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int):
    if status != AH_OK:
        raise AhError(status, load().ah_last_error().decode())


# ---- same-name wrappers of the C ABI -------------------------------------------------
def ah_abi_version() -> int:
    return load().ah_abi_version()


def ah_last_error() -> str:
    return load().ah_last_error().decode()


def ah_config_default(N: int) -> ah_config:
    c = ah_config()
    load().ah_config_default(ctypes.byref(c), N)
    return c


def ah_create(N, dx, dt, era, s, lambda0, e0, seed) -> int:
    h = load().ah_create(N, dx, dt, era, s, lambda0, e0, seed)
    if not h:
        raise AhError(-1, ah_last_error())
    return h


def ah_create_ex(cfg: ah_config) -> int:
    h = ctypes.c_void_p()
    _check(load().ah_create_ex(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def ah_step(h, nsteps: int):
    _check(load().ah_step(h, nsteps))


def ah_observables(h, check_finite: bool = True) -> dict:
    o = ah_obs()
    st = load().ah_observables(h, ctypes.byref(o))
    if st != AH_OK and not (st == AH_ERR_NONFINITE and not check_finite):
        _check(st)
    return o.as_dict()


def ah_observables_start(h):
    _check(load().ah_observables_start(h))


def ah_observables_finish(h, check_finite: bool = True) -> dict:
    o = ah_obs()
    st = load().ah_observables_finish(h, ctypes.byref(o))
    if st != AH_OK and not (st == AH_ERR_NONFINITE and not check_finite):
        _check(st)
    return o.as_dict()


def ah_observables_box(h, x0, y0, z0, nx, ny, nz) -> dict:
    o = ah_obs()
    _check(load().ah_observables_box(h, x0, y0, z0, nx, ny, nz, ctypes.byref(o)))
    return o.as_dict()


def ah_get_fields(h, x0, y0, z0, nx, ny, nz) -> np.ndarray:
    out = np.empty((10, nz, ny, nx), dtype=np.float64)
    _check(load().ah_get_fields(h, x0, y0, z0, nx, ny, nz, out.ctypes.data))
    return out


def ah_set_fields(h, fields: np.ndarray, step: int = 0):
    f = np.ascontiguousarray(fields, dtype=np.float64)
    _check(load().ah_set_fields(h, f.ctypes.data, step))


def ah_set_stream(h, stream_ptr: int | None):
    _check(load().ah_set_stream(h, stream_ptr or None))


def ah_sync(h):
    _check(load().ah_sync(h))


def ah_get_step(h) -> int:
    return load().ah_get_step(h)


def ah_get_tau(h) -> float:
    return load().ah_get_tau(h)


def ah_get_info(h) -> dict:
    i = ah_info()
    _check(load().ah_get_info(h, ctypes.byref(i)))
    d = {n: getattr(i, n) for n, _ in i._fields_}
    d["variant_name"] = d["variant_name"].decode()
    return d


def ah_variant_count(precision: int) -> int:
    return load().ah_variant_count(precision)


def ah_set_variant(h, variant: int):
    _check(load().ah_set_variant(h, variant))


def ah_autotune(h, trial_steps: int = 3) -> int:
    v = ctypes.c_int32(-1)
    _check(load().ah_autotune(h, trial_steps, ctypes.byref(v)))
    return v.value


def ah_destroy(h):
    if h:
        load().ah_destroy(h)


class ah_sums(ctypes.Structure):
    _fields_ = [("sums", ctypes.c_double * 16), ("gauss_max", ctypes.c_double), ("max_abs_theta", ctypes.c_double),
                ("wind_abs_plane", ctypes.c_int64 * 3), ("wind_plane", ctypes.c_int64 * 3),
                ("n_pierced", ctypes.c_int64), ("nonfinite", ctypes.c_int64)]


def ah_observables_noalloc(field_ptrs, N: int, cfg: ah_config, step: int, d_sums_ptr: int, stream_ptr=None):
    """Diagnostics of an FP32 state in caller-owned device buffers (10 device
    pointers), written as an ah_sums to the device pointer d_sums_ptr; no device
    allocation.  Enqueued on stream_ptr; synchronise before reading the sums."""
    arr = (ctypes.c_void_p * 10)(*[int(p) for p in field_ptrs])
    _check(load().ah_observables_noalloc(arr, N, ctypes.byref(cfg), step, d_sums_ptr, stream_ptr or None))


def _windows(wins, lattice_of=None):
    """ah_window array and the numpy buffers it points to, from (x0, y0, z0, nx, ny, nz)
    boxes (with a leading lattice index when lattice_of is None)."""
    arr = (ah_window * max(1, len(wins)))()
    bufs = []
    for k, w in enumerate(wins):
        lat, box = (w[0], w[1:]) if lattice_of is None else (lattice_of, w)
        x0, y0, z0, nx, ny, nz = box
        b = np.empty((10, nz, ny, nx), dtype=np.float64)
        bufs.append(b)
        arr[k] = ah_window(lat, x0, y0, z0, nx, ny, nz, b.ctypes.data)
    return arr, bufs


def ah_batch_run(cfgs, flags: int = 0, series_cap: int = 64):
    """Run a batch of FP32 lattices to their ends; returns (series, stats): series[i]
    is the list of observable dicts of lattice i (step 0, every diag_every, end)."""
    n = len(cfgs)
    arr = (ah_config * n)(*cfgs)
    series = (ah_obs * (n * series_cap))()
    lens = (ctypes.c_int64 * n)()
    st = ah_batch_stats()
    _check(load().ah_batch_run(arr, n, flags, series, series_cap, lens, ctypes.byref(st)))
    out = [[series[i * series_cap + k].as_dict() for k in range(min(lens[i], series_cap))] for i in range(n)]
    return out, {k: getattr(st, k) for k, _ in st._fields_}


def ah_batch_run_ex(cfgs, windows=(), flags: int = 0, series_cap: int = 64):
    """ah_batch_run plus read-back of final-state windows: `windows` holds
    (lattice, x0, y0, z0, nx, ny, nz) tuples; returns (series, stats, fields) with
    fields[k] the (10, nz, ny, nx) FP64 array of window k."""
    n = len(cfgs)
    arr = (ah_config * n)(*cfgs)
    series = (ah_obs * (n * series_cap))()
    lens = (ctypes.c_int64 * n)()
    st = ah_batch_stats()
    warr, bufs = _windows(list(windows))
    _check(load().ah_batch_run_ex(arr, n, flags, series, series_cap, lens, ctypes.byref(st), warr, len(bufs)))
    out = [[series[i * series_cap + k].as_dict() for k in range(min(lens[i], series_cap))] for i in range(n)]
    return out, {k: getattr(st, k) for k, _ in st._fields_}, bufs


class Server:
    """Continuous-batching server (ah_server_*): submit runs, poll their results."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, flags: int = 0):
        h = ctypes.c_void_p()
        _check(load().ah_server_create(hbm_budget_bytes, max_slots, flags, ctypes.byref(h)))
        self.h = h.value
        self._keep = {}

    def submit(self, cfg: ah_config) -> int:
        rid = ctypes.c_uint64()
        _check(load().ah_server_submit(self.h, ctypes.byref(cfg), ctypes.byref(rid)))
        return rid.value

    def submit_ex(self, cfg: ah_config, windows=()):
        """Queue a run whose final-state windows ((x0, y0, z0, nx, ny, nz) boxes) are
        written when it completes; returns (request id, list of (10, nz, ny, nx)
        arrays), valid once poll() reports the request done."""
        rid = ctypes.c_uint64()
        warr, bufs = _windows(list(windows), lattice_of=0)
        _check(load().ah_server_submit_ex(self.h, ctypes.byref(cfg), warr, len(bufs), ctypes.byref(rid)))
        self._keep[rid.value] = (warr, bufs)      # the library writes into these buffers later
        return rid.value, bufs

    def poll(self, rid: int):
        """None while queued or running, else (obs dict, t_submit, t_done)."""
        o, ts, td = ah_obs(), ctypes.c_double(), ctypes.c_double()
        st = load().ah_server_poll(self.h, rid, ctypes.byref(o), ctypes.byref(ts), ctypes.byref(td))
        if st == AH_ERR_BUSY:
            return None
        _check(st)
        return o.as_dict(), ts.value, td.value

    def cancel(self, rid: int):
        _check(load().ah_server_cancel(self.h, rid))

    def stats(self) -> dict:
        s = ah_server_stats()
        _check(load().ah_server_stats_get(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if self.h:
            load().ah_server_destroy(self.h)
            self.h = None
            self._keep = {}

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience ------------------------------------------------------------------
def config(N: int, **kw) -> ah_config:
    """ah_config with the library defaults for N, fields overridden by keyword."""
    c = ah_config_default(N)
    if "tau_end" not in kw and "dx" in kw:
        kw["tau_end"] = N * kw["dx"] / 2.0
    if "tau_ref" not in kw:
        kw["tau_ref"] = kw.get("tau_end", c.tau_end)
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


class Sim:
    """Owning wrapper of one simulation handle."""

    def __init__(self, N: int, **kw):
        self.cfg = config(N, **kw)
        self.h = ah_create_ex(self.cfg)
        self.N = N

    def step(self, n: int = 1):
        ah_step(self.h, n)
        return self

    def observables(self, check_finite=True) -> dict:
        return ah_observables(self.h, check_finite)

    def observables_start(self):
        ah_observables_start(self.h)
        return self

    def observables_finish(self, check_finite=True) -> dict:
        return ah_observables_finish(self.h, check_finite)

    def observables_box(self, x0, y0, z0, nx, ny, nz) -> dict:
        return ah_observables_box(self.h, x0, y0, z0, nx, ny, nz)

    def fields(self, x0=0, y0=0, z0=0, nx=None, ny=None, nz=None) -> np.ndarray:
        N = self.N
        return ah_get_fields(self.h, x0, y0, z0, nx or N, ny or N, nz or N)

    def set_fields(self, f: np.ndarray, step: int = 0):
        ah_set_fields(self.h, f, step)

    def set_variant(self, variant: int):
        ah_set_variant(self.h, variant)
        return self

    def autotune(self, trial_steps: int = 3) -> int:
        return ah_autotune(self.h, trial_steps)

    def sync(self):
        ah_sync(self.h)

    @property
    def n(self) -> int:
        return ah_get_step(self.h)

    @property
    def info(self) -> dict:
        return ah_get_info(self.h)

    def close(self):
        if self.h:
            ah_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
