"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

This module holds none of the method's arithmetic: it only draws random or
analytic field configurations (numpy, FP64) in the (10, M, M, M) layout
(phi.re, phi.im, Pi.re, Pi.im, theta_1..3, E_1..3; index [c, z, y, x]).
"""
from __future__ import annotations

import numpy as np


def random_state(M: int, seed: int, phi_amp=1.0, pi_amp=0.5, th_amp=0.4, e_amp=0.3) -> np.ndarray:
    """Generic random state: every term of both kicks is non-zero from step 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = np.empty((10, M, M, M), dtype=np.float64)
    f[0:2] = rng.uniform(-phi_amp, phi_amp, size=(2, M, M, M))
    f[2:4] = rng.uniform(-pi_amp, pi_amp, size=(2, M, M, M))
    f[4:7] = rng.uniform(-th_amp, th_amp, size=(3, M, M, M))
    f[7:10] = rng.uniform(-e_amp, e_amp, size=(3, M, M, M))
    return f


def random_angles(M: int, seed: int, lo=0.0, hi=2 * np.pi) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(M, M, M))


def coords(M: int):
    """Integer site coordinates (z, y, x) broadcastable to (M, M, M)."""
    k, j, i = np.meshgrid(np.arange(M), np.arange(M), np.arange(M), indexing="ij")
    return i, j, k


def straight_strings(M: int, axis: int = 2, x0=0.3, y0=0.7) -> np.ndarray:
    """phi = s_a + i s_b, normalised to |phi| = 1, with s_a = sin(2 pi (a - a0)/M)
    and s_b = sin(2 pi (b - b0)/M) over the two coordinates transverse to `axis`;
    the zeros form four straight strings along `axis` with windings +1, -1, -1, +1.
    The offsets are off-lattice so that no site sits on a zero.  Pi = theta = E = 0."""
    i, j, k = coords(M)
    c = [i, j, k]
    tr = [d for d in range(3) if d != axis]
    sa = np.sin(2 * np.pi * (c[tr[0]] - x0) / M)
    sb = np.sin(2 * np.pi * (c[tr[1]] - y0) / M)
    r = np.sqrt(sa * sa + sb * sb)
    f = np.zeros((10, M, M, M))
    f[0] = sa / r
    f[1] = sb / r
    return f
