"""Plain FP64 CPU oracle for the lattice Abelian-Higgs leapfrog and its diagnostics.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers; the product library
never imports this package.  The arithmetic lives in ``ah_oracle.c`` (plain C,
FP64, one site at a time); this module compiles it with gcc and marshals numpy
arrays through ctypes.  It shares no code with the CUDA library.

Field arrays have shape (10, M, M, M) (component, z, y, x) with components
phi.re, phi.im, Pi.re, Pi.im, theta_1..3, E_1..3 (Sec. 2 of arXiv:1809.00995).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ah_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libah_oracle.so")
_lock = threading.Lock()
_lib = None

MINKOWSKI, RADIATION, MATTER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ah_oracle.c into oracle/lib/libah_oracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("era", ctypes.c_int32), ("flags", ctypes.c_int32), ("s", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("e0", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tau0", ctypes.c_double), ("tau_ref", ctypes.c_double), ("seed", ctypes.c_uint64)]


class _Diag(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_double) for n in (
        "sum_L", "sum_rho", "sum_p", "sum_K", "sum_G2", "sum_V", "sum_Eel", "sum_B",
        "sum_KV", "sum_G2V", "sum_KL", "sum_G2L", "sum_pL", "sum_rhoL",
        "sum_gauss2", "max_gauss", "sum_gscale2", "max_abs_theta")]
        + [("sum_abs_W", ctypes.c_int64), ("n_pierced", ctypes.c_int64),
           ("sum_abs_W_plane", ctypes.c_int64 * 3), ("sum_W_plane", ctypes.c_int64 * 3),
           ("nonfinite", ctypes.c_int64), ("n_sites", ctypes.c_int64)])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(_Params)
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.aho_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            lib.aho_site_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.aho_site_uniform.restype = ctypes.c_double
            lib.aho_scale_factor.argtypes = [P, ctypes.c_double]
            lib.aho_scale_factor.restype = ctypes.c_double
            lib.aho_init_box.argtypes = [P, dp, i64, i64, i64, i64]
            lib.aho_step.argtypes = [P, dp, i64, i64]
            lib.aho_step.restype = ctypes.c_int
            lib.aho_evolve.argtypes = [P, dp, i64, i64, i64]
            lib.aho_evolve.restype = ctypes.c_int
            lib.aho_diag.argtypes = [P, dp, i64, i64, i64, i64, i64, i64, i64, i64,
                                     ctypes.POINTER(_Diag)]
            lib.aho_energy.argtypes = [P, dp, i64, i64]
            lib.aho_energy.restype = ctypes.c_double
            lib.aho_gauge_transform.argtypes = [dp, i64, dp]
            lib.aho_windings.argtypes = [dp, i64, ctypes.POINTER(ctypes.c_int8)]
            _lib = lib
    return _lib


@dataclass
class Params:
    """Run parameters (Sec. 2): lattice side N, spacing dx, step dt, era, exponent s,
    couplings lambda0, e0, vev sigma, start time tau0, normalisation a(tau_ref) = 1, seed."""
    N: int
    dx: float = 0.5
    dt: float = 0.1
    era: int = RADIATION
    s: float = 0.0
    lambda0: float = 2.0
    e0: float = 1.0
    sigma: float = 1.0
    tau0: float = 1.0
    tau_ref: float | None = None   # default: tau_end = N dx / 2
    seed: int = 1
    wrap_theta: bool = False       # compact link phases: theta kept in [-pi, pi]
    core_growth: bool = False      # exponent s before tau_ref, 1 from tau_ref on (Eq. 7)

    @property
    def tau_end(self) -> float:
        return self.N * self.dx / 2.0

    def c(self) -> _Params:
        tr = self.tau_end if self.tau_ref is None else self.tau_ref
        flags = (1 if self.wrap_theta else 0) | (2 if self.core_growth else 0)
        return _Params(self.N, self.dx, self.dt, self.era, flags, self.s, self.lambda0, self.e0,
                       self.sigma, self.tau0, tr, self.seed)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def philox4x32_10(ctr, key):
    """Philox-4x32-10 block function (Salmon et al., SC'11)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.aho_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def site_uniform(seed: int, idx: int) -> float:
    return _load().aho_site_uniform(seed, idx)


def scale_factor(p: Params, tau: float) -> float:
    cp = p.c()
    return _load().aho_scale_factor(ctypes.byref(cp), tau)


def new_fields(M: int) -> np.ndarray:
    return np.zeros((10, M, M, M), dtype=np.float64)


def init(p: Params, M: int | None = None, origin=(0, 0, 0)) -> np.ndarray:
    """Random-phase initial state of the M^3 box at global origin (x0, y0, z0)."""
    M = p.N if M is None else M
    f = new_fields(M)
    cp = p.c()
    _load().aho_init_box(ctypes.byref(cp), _dp(f), M, *[int(o) for o in origin])
    return f


def evolve(p: Params, f: np.ndarray, n0: int, nsteps: int) -> np.ndarray:
    """Advance f (in place) from step n0 by nsteps leapfrog steps."""
    M = f.shape[1]
    cp = p.c()
    rc = _load().aho_evolve(ctypes.byref(cp), _dp(f), M, n0, nsteps)
    if rc != 0:
        raise MemoryError("oracle evolve failed")
    return f


def diag_sums(p: Params, f: np.ndarray, n: int, box=None) -> dict:
    """Raw FP64 diagnostic sums at step n over a sub-box (x0, y0, z0, nx, ny, nz)."""
    M = f.shape[1]
    box = (0, 0, 0, M, M, M) if box is None else box
    d = _Diag()
    cp = p.c()
    _load().aho_diag(ctypes.byref(cp), _dp(f), M, n, *[int(b) for b in box], ctypes.byref(d))
    out = {}
    for name, _ in _Diag._fields_:
        v = getattr(d, name)
        out[name] = list(v) if name.endswith("_plane") else v
    return out


def observables(p: Params, f: np.ndarray, n: int, box=None) -> dict:
    """Network observables at step n (Eqs. defXiV2, defR, 9, defEoS):
    xi_L = sqrt(-mu / mean L) with mu = 2 pi sigma^2; xi_W = sqrt(V / l_W) with
    l_W = (pi/6) dx sum|W|; <v^2>_X = 2R/(1+R), R = sum K X / sum |D phi|^2 X for
    X = V, L; <v^2>_omega = (1 + 3 sum pL / sum rho L)/2; Gauss residual."""
    d = diag_sums(p, f, n, box)
    ns = d["n_sites"]
    mu = 2.0 * math.pi * p.sigma ** 2
    with np.errstate(all="ignore"):
        Lbar = d["sum_L"] / ns
        o = dict(d)
        o["L_mean"] = Lbar
        o["xi_L"] = float(np.sqrt(np.float64(-mu) / np.float64(Lbar)))
        lw = math.pi / 6.0 * p.dx * d["sum_abs_W"]
        o["xi_W"] = float(np.sqrt(np.float64(ns * p.dx ** 3) / np.float64(lw)))
        RV = np.float64(d["sum_KV"]) / np.float64(d["sum_G2V"])
        RL = np.float64(d["sum_KL"]) / np.float64(d["sum_G2L"])
        o["R_V"], o["R_L"] = float(RV), float(RL)
        o["v2_V"] = float(2 * RV / (1 + RV))
        o["v2_L"] = float(2 * RL / (1 + RL))
        o["p_over_rho_L"] = float(np.float64(d["sum_pL"]) / np.float64(d["sum_rhoL"]))
        o["v2_omega"] = 0.5 * (1.0 + 3.0 * o["p_over_rho_L"])
        o["gauss_rms"] = math.sqrt(d["sum_gauss2"] / ns)
        o["gauss_max"] = d["max_gauss"]
        o["gauss_rel"] = float(np.sqrt(np.float64(d["sum_gauss2"]) / np.float64(d["sum_gscale2"])))
        o["energy"] = d["sum_rho"] * p.dx ** 3
    return o


def energy(p: Params, f: np.ndarray, n: int) -> float:
    cp = p.c()
    return _load().aho_energy(ctypes.byref(cp), _dp(f), f.shape[1], n)


def gauge_transform(f: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """In-place lattice gauge transform by angles alpha (shape (M, M, M))."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    _load().aho_gauge_transform(_dp(f), f.shape[1], _dp(alpha))
    return f


def windings(f: np.ndarray) -> np.ndarray:
    """Per-site winding numbers, shape (3, M, M, M), orientations 12, 13, 23."""
    M = f.shape[1]
    w = np.zeros((3, M, M, M), dtype=np.int8)
    _load().aho_windings(_dp(f), M, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return w
