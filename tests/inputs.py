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


_BPS_CACHE = {}


def bps_profile(R=16.0):
    """Radial profile of the unit-winding Nielsen-Olesen string at critical
    coupling (lambda0 = 2 e0^2, e0 = sigma = 1): phi = f(r) e^{i alpha},
    A = a(r) grad(alpha) / e0, from the first-order Bogomolny equations
    f' = (1 - a) f / r, a' = r (1 - f^2), f(0) = a(0) = 0, f, a -> 1, solved by
    shooting on f'(0) with scipy's DOP853-class integrator.  Its tension is
    2 pi sigma^2.  Returns a vectorised r -> (f, a) (the vacuum beyond the last
    radius where the shot trajectory is still converging)."""
    if R in _BPS_CACHE:
        return _BPS_CACHE[R]
    from scipy.integrate import solve_ivp

    def rhs(r, y):
        return [(1.0 - y[1]) * y[0] / r, r * (1.0 - y[0] * y[0])]

    r0 = 1e-5

    def shoot(c):
        ev = lambda r, y: y[0] - 1.0          # noqa: E731
        ev.terminal = True
        return solve_ivp(rhs, (r0, R), [c * r0, r0 * r0 / 2.0], method="DOP853", rtol=1e-12, atol=1e-14,
                         events=[ev], dense_output=True)

    lo, hi = 0.5, 1.2                          # f'(0): too small turns f down, too large overshoots 1
    for _ in range(60):
        c = 0.5 * (lo + hi)
        if shoot(c).t_events[0].size:
            hi = c
        else:
            lo = c
    sol = shoot(lo)
    rs = np.linspace(r0, sol.t[-1], 20001)
    one_minus_f = 1.0 - sol.sol(rs)[0]
    up = np.nonzero(np.diff(one_minus_f) > 0)[0]
    rcut = rs[up[0]] if up.size else rs[-1]

    def fa(r):
        r = np.asarray(r, dtype=np.float64)
        f, a = np.ones_like(r), np.ones_like(r)
        m = r < rcut
        rr = np.maximum(r[m], r0)
        v = sol.sol(rr.ravel())
        near = r[m] < r0
        f[m] = np.where(near, lo * r[m], v[0].reshape(rr.shape))
        a[m] = np.where(near, r[m] * r[m] / 2.0, v[1].reshape(rr.shape))
        return f, a

    _BPS_CACHE[R] = (fa, lo)
    return fa, lo


def bps_string(N: int, dx: float, off=(0.31, 0.17)) -> np.ndarray:
    """A static straight BPS string along z through the middle of an N^3 periodic
    lattice (e0 = sigma = 1): phi = f(r) e^{i alpha} at the sites, theta_1,2 the
    link phases -int a(r) d(alpha) along each link (12-point Gauss-Legendre, so
    that U phi^{x+i} ~ phi^x far from the core), plus on the links that wrap
    around the box the pure-gauge jump of alpha between the two images;
    theta_3 = Pi = E = 0.  The core sits off-lattice at offset `off` (in
    spacings) from the centre of the middle plaquette."""
    fa, _ = bps_profile()
    xc, yc = (N / 2 - 0.5 + off[0]) * dx, (N / 2 - 0.5 + off[1]) * dx
    ii = np.arange(N) * dx
    X, Y = np.meshgrid(ii, ii, indexing="xy")          # [y, x]
    alpha = np.arctan2(Y - yc, X - xc)
    f, _ = fa(np.hypot(X - xc, Y - yc))
    gx, gw = np.polynomial.legendre.leggauss(12)
    th = []
    for d in range(2):
        ex, ey = (1.0, 0.0) if d == 0 else (0.0, 1.0)
        acc = np.zeros((N, N))
        for t, w in zip(0.5 * (gx + 1.0), 0.5 * gw):
            px, py = X + t * dx * ex - xc, Y + t * dx * ey - yc
            r2 = px * px + py * py
            _, a = fa(np.sqrt(r2))
            acc += w * a * (px * dx * ey - py * dx * ex) / r2      # a(r) d(alpha)/dt
        jump = np.arctan2(Y + dx * ey - yc, X + dx * ex - xc) - np.roll(alpha, -1, axis=1 - d)
        th.append(jump - acc)
    out = np.zeros((10, N, N, N))
    out[0] = (f * np.cos(alpha))[None]
    out[1] = (f * np.sin(alpha))[None]
    out[4] = th[0][None]
    out[5] = th[1][None]
    return out
