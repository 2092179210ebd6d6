"""Pins of the FP64 CPU oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: published
Philox test vectors, closed-form solutions of the linearised lattice equations,
exact conservation laws and symmetries of the scheme, second-order convergence
to an independent high-accuracy ODE solution, and analytically placed strings.
A plausible slip in the oracle (a dropped term, a wrong sign, index or
coefficient, a transposed operand) breaks at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from inputs import bps_string, coords, random_angles, random_state, straight_strings

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox / init
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_init_random_phase_and_window_consistency():
    from scipy import stats
    p = O.Params(N=16, seed=5, sigma=1.3)
    f = O.init(p)
    mod = np.hypot(f[0], f[1])
    assert np.max(np.abs(mod - 1.3)) < 1e-14
    assert not np.any(f[2:])
    u = (np.arctan2(f[1], f[0]) / (2 * np.pi)) % 1.0
    assert stats.kstest(u.ravel(), "uniform").pvalue > 1e-4
    # a window whose box wraps across the periodic seam holds the same sites
    w = O.init(p, M=6, origin=(13, 2, 7))
    idx = [(np.arange(6) + o) % 16 for o in (13, 2, 7)]
    sub = f[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    assert np.array_equal(w, sub)
    # distinct seeds give distinct phases
    g = O.init(O.Params(N=16, seed=6, sigma=1.3))
    assert np.mean(np.abs(g[0] - f[0]) > 1e-3) > 0.9


def test_site_uniform_matches_its_exact_definition():
    """The uniform behind each initial phase (Sec. 2: alpha = 2 pi u, u from
    Philox) equals the golden values that tests/golden/make_site_uniform.py
    computed in exact rational arithmetic from the known-answer-pinned Philox
    words: key = seed, counter = (0, 0, index), u = (w0 2^21 + w1 >> 11) 2^-53.
    A slip in a shift, the word order, the counter or key layout (indices and
    seeds past 2^32 included) or the scale changes these bits."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "site_uniform.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for seed, idx, u in rows:
        assert O.site_uniform(int(seed), int(idx)) == float.fromhex(u), (seed, idx)
    # the initial state uses it: phi at a site is sigma e^{2 pi i u}
    p = O.Params(N=16, seed=1, sigma=1.0)
    f = O.init(p)
    u0 = float.fromhex(rows[0][2])
    assert int(rows[0][0]) == 1 and int(rows[0][1]) == 0
    assert abs(f[0, 0, 0, 0] - math.cos(2 * math.pi * u0)) < 1e-15
    assert abs(f[1, 0, 0, 0] - math.sin(2 * math.pi * u0)) < 1e-15


# ---------------------------------------------------------------- closed forms
def _leapfrog_amplitude(omega, dt, n):
    """Exact discrete solution of A_{n+1} - 2A_n + A_{n-1} = -dt^2 w^2 A_n with
    A_{-1} = A_0 = 1 (momentum zero at n = -1/2)."""
    Om = 2.0 * math.asin(dt * omega / 2.0) / dt
    return math.cos(Om * (n + 0.5) * dt) / math.cos(Om * dt / 2.0)


@pytest.mark.parametrize("gauge", [False, True])
def test_scalar_wave_closed_form(gauge):
    """Minkowski, lambda = 0, theta = 0, real phi = eps cos(k.x): the current vanishes,
    E = theta = 0 stay, and phi follows the lattice Klein-Gordon dispersion
    w^2 = (4/dx^2) sum_j sin^2(k_j dx / 2).  With gauge=True the same solution is
    gauge transformed by random angles first (theta != 0) and transformed back."""
    N, m, eps = 12, (1, 2, 3), 0.3
    p = O.Params(N=N, era=O.MINKOWSKI, lambda0=0.0, dx=0.5, dt=0.1)
    i, j, k = coords(N)
    ph = 2 * np.pi * (m[0] * i + m[1] * j + m[2] * k) / N
    f = O.new_fields(N)
    f[0] = eps * np.cos(ph)
    omega = math.sqrt(4 / p.dx ** 2 * sum(math.sin(math.pi * mj / N) ** 2 for mj in m))
    alpha = random_angles(N, 11)
    if gauge:
        O.gauge_transform(f, alpha)
        assert np.max(np.abs(f[4:7])) > 0.5
    nsteps = 40
    O.evolve(p, f, 0, nsteps)
    if gauge:
        O.gauge_transform(f, -alpha)
    A = _leapfrog_amplitude(omega, p.dt, nsteps)
    assert np.max(np.abs(f[0] - eps * A * np.cos(ph))) < 1e-12
    assert np.max(np.abs(f[1])) < 1e-12
    assert np.max(np.abs(f[7:10])) < 1e-12
    assert np.max(np.abs(f[4:7])) < 1e-12


def test_transverse_gauge_wave_closed_form():
    """phi = 0, Minkowski, small transverse link wave theta_i = eps_i cos(k.x + k_i dx/2)
    with sum_i eps_i sin(k_i dx/2) = 0: the lattice curl-curl acts as -w^2 with the
    same lattice dispersion, through every plaquette term including the diagonal
    neighbours x+i-j.  Valid to O(eps^2) relative."""
    N, m = 12, np.array([1, 2, 3])
    p = O.Params(N=N, era=O.MINKOWSKI, dx=0.5, dt=0.1)
    s = np.sin(np.pi * m / N)
    pol = np.cross(s, [0.3, -0.7, 0.2])
    pol *= 1e-5 / np.linalg.norm(pol)
    i, j, k = coords(N)
    ph = 2 * np.pi * (m[0] * i + m[1] * j + m[2] * k) / N
    f = O.new_fields(N)
    init = [pol[d] * np.cos(ph + np.pi * m[d] / N) for d in range(3)]
    for d in range(3):
        f[4 + d] = init[d]
    omega = math.sqrt(4 / p.dx ** 2 * float(np.sum(s * s)))
    nsteps = 37
    O.evolve(p, f, 0, nsteps)
    A = _leapfrog_amplitude(omega, p.dt, nsteps)
    for d in range(3):
        assert np.max(np.abs(f[4 + d] - A * init[d])) < 1e-8 * np.max(np.abs(pol))
    assert abs(A) < 0.9  # the wave really moved


def test_uniform_mode_damping_closed_forms():
    """Uniform fields, lambda = 0: the Laplacian, current and curl vanish, so the kicks
    reduce to the damping factors: a_{n+1/2}^2 Pi^{n+1/2} = a_{-1/2}^2 Pi^{-1/2} (theta = 0)
    and E^{n+1/2} / e_{n+1/2}^2 = E^{-1/2} / e_{-1/2}^2 (phi = Pi = 0) exactly, with the
    Eq. 7 couplings and the half-step a evaluated at tau_n +- dt/2."""
    p = O.Params(N=4, era=O.RADIATION, s=0.5, lambda0=0.0, tau_ref=3.0)
    n = 25
    a = lambda t: t / 3.0
    am, ap = a(p.tau0 - p.dt / 2), a(p.tau0 + (n - 0.5) * p.dt)
    f = O.new_fields(4)
    f[0], f[1], f[2], f[3] = 0.3, -0.2, 0.1, 0.05
    O.evolve(p, f, 0, n)
    assert abs(f[2, 0, 0, 0] - 0.1 * am ** 2 / ap ** 2) < 1e-15
    assert abs(f[3, 1, 0, 2] - 0.05 * am ** 2 / ap ** 2) < 1e-15
    pis = [0.1 * am ** 2 / a(p.tau0 + (q + 0.5) * p.dt) ** 2 for q in range(n)]
    assert abs(f[0, 3, 3, 3] - (0.3 + p.dt * sum(pis))) < 1e-14
    assert not np.any(f[4:10])
    g = O.new_fields(4)
    g[7], g[8], g[9] = 0.1, 0.2, -0.3
    g[4], g[5], g[6] = 0.2, -0.1, 0.3
    O.evolve(p, g, 0, n)
    e2 = lambda aa: aa ** (2 * (p.s - 1))
    for d, e0 in enumerate((0.1, 0.2, -0.3)):
        assert abs(g[7 + d, 1, 2, 3] - e0 * e2(ap) / e2(am)) < 1e-15
    assert not np.any(g[0:4])


def _uniform_ode(p, y0, t0, t1):
    """Continuous-time equations of the model for spatially uniform phi and theta_i on
    the lattice (Eq. 1 with Eq. 7 couplings in conformal time):
      (a^2 phi')' = (a^2/dx^2) sum_j (2 cos theta_j - 2) phi - a^4 (lambda/2)(|phi|^2 - sigma^2) phi
      (theta_i' / e^2)' = 2 a^2 Im[conj(phi) e^{-i theta_i} phi] = -2 a^2 |phi|^2 sin theta_i
    integrated to rtol 1e-13 with scipy's DOP853."""
    from scipy.integrate import solve_ivp
    alpha = {0: 0, 1: 1, 2: 2}[p.era]
    tr = p.tau_ref

    def rhs(t, y):
        a = (t / tr) ** alpha
        da = alpha * (t / tr) ** (alpha - 1) / tr if alpha else 0.0
        H = da / a
        e2 = p.e0 ** 2 * a ** (2 * (p.s - 1))
        de2 = e2 * 2 * (p.s - 1) * H
        lam = p.lambda0 * a ** (2 * (p.s - 1))
        ph = y[0] + 1j * y[1]
        dph = y[2] + 1j * y[3]
        th, dth = y[4:7], y[7:10]
        lap = sum(2 * math.cos(t_) - 2 for t_ in th) / p.dx ** 2 * ph
        pot = a ** 2 * lam / 2 * (abs(ph) ** 2 - p.sigma ** 2) * ph
        ddph = -2 * H * dph + lap - pot
        ddth = de2 / e2 * dth - 2 * a ** 2 * e2 * abs(ph) ** 2 * np.sin(th)
        return np.concatenate([[dph.real, dph.imag, ddph.real, ddph.imag], dth, ddth])

    sol = solve_ivp(rhs, (t0, t1), y0, method="DOP853", rtol=1e-13, atol=1e-15)
    return sol.y[:, -1]


@pytest.mark.parametrize("era,s", [(O.RADIATION, 0.0), (O.MATTER, 1.0), (O.RADIATION, -0.5)])
def test_uniform_mode_second_order_convergence(era, s):
    """The leapfrog (Eqs. up_pi .. up_A) must converge at second order in dt to the
    continuous-time equations of uniform fields; a wrong time-centring of any
    coefficient (a_n vs a_{n+1/2}, an averaged half-step a) makes it first order."""
    p0 = O.Params(N=4, era=era, s=s, lambda0=2.0, e0=1.0, tau_ref=4.0, tau0=1.0)
    y_init = np.array([0.6, 0.3, 0.1, -0.2, 0.3, -0.5, 1.0, 0.2, 0.1, -0.1])
    T = 2.0
    ref = _uniform_ode(p0, y_init, p0.tau0, p0.tau0 + T)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        p = O.Params(**{**p0.__dict__, "dt": dt})
        back = _uniform_ode(p, y_init, p.tau0, p.tau0 - dt / 2)   # momenta at tau0 - dt/2
        f = O.new_fields(4)
        f[0], f[1] = y_init[0], y_init[1]
        f[2], f[3] = back[2], back[3]
        for d in range(3):
            f[4 + d] = y_init[4 + d]
            f[7 + d] = back[7 + d]
        n = int(round(T / dt))
        O.evolve(p, f, 0, n)
        got = np.array([f[0, 0, 0, 0], f[1, 0, 0, 0]] + [f[4 + d, 0, 0, 0] for d in range(3)])
        want = np.array([ref[0], ref[1], ref[4], ref[5], ref[6]])
        errs.append(np.max(np.abs(got - want)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs
    assert errs[2] < 1e-3


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("era,s", [(O.RADIATION, 0.0), (O.MATTER, 1.0), (O.MINKOWSKI, 0.0)])
def test_gauss_law_conserved(era, s):
    """The discrete Gauss residual is conserved exactly by the kicks and drifts:
    zero from the random-phase init, and unchanged site by site from a random state."""
    p = O.Params(N=10, era=era, s=s, seed=3, tau_ref=5.0 if s else None)
    f = O.init(p)
    O.evolve(p, f, 0, 60)
    o = O.observables(p, f, 60)
    assert o["gauss_max"] < 1e-13
    assert o["sum_K"] > 1.0 and o["sum_Eel"] > 0.01   # the fields did evolve
    g = random_state(9, 21)
    o0 = O.observables(p, g, 0)
    O.evolve(p, g, 0, 30)
    o1 = O.observables(p, g, 30)
    assert o0["gauss_rms"] > 0.01
    assert abs(o1["gauss_rms"] - o0["gauss_rms"]) < 1e-12 * o0["gauss_rms"]
    assert abs(o1["gauss_max"] - o0["gauss_max"]) < 1e-12 * o0["gauss_max"]


def test_gauge_invariance():
    """Observables and windings are unchanged by a random lattice gauge transform,
    and the evolution commutes with it."""
    p = O.Params(N=8, era=O.RADIATION, s=0.0, seed=9)
    f = O.init(p)
    O.evolve(p, f, 0, 6)
    g = f.copy()
    alpha = random_angles(8, 4)
    O.gauge_transform(g, alpha)
    of, og = O.observables(p, f, 6), O.observables(p, g, 6)
    for k in ("sum_L", "sum_rho", "sum_p", "sum_KV", "sum_G2V", "sum_pL", "sum_B", "sum_gauss2"):
        assert abs(of[k] - og[k]) <= 1e-12 * max(1.0, abs(of[k])), k
    assert np.array_equal(O.windings(f), O.windings(g))
    assert of["sum_abs_W"] > 0
    O.evolve(p, f, 6, 10)
    O.evolve(p, g, 6, 10)
    O.gauge_transform(g, -alpha)
    assert np.max(np.abs(f - g)) < 1e-11
    # a large gauge shift theta -> theta + 2 pi m changes nothing physical
    h = f.copy()
    h[4:7] += 2 * np.pi * np.random.Generator(np.random.PCG64(2)).integers(-2, 3, size=(3, 8, 8, 8))
    assert np.array_equal(O.windings(h), O.windings(f))


def test_coupling_rescaling_symmetry():
    """For any s the scheme is exactly invariant under a -> c a with
    lambda0 -> lambda0 c^{-2s} and e0 -> e0 c^{-s}; this fixes the total power of a
    in every kick coefficient (Eqs. up_pi, up_E with Eq. 7)."""
    for s in (0.0, 1.0, 0.5):
        c = 2.0
        pa = O.Params(N=6, era=O.RADIATION, s=s, tau_ref=8.0)
        pb = O.Params(N=6, era=O.RADIATION, s=s, tau_ref=8.0 / c,
                      lambda0=2.0 * c ** (-2 * s), e0=c ** (-s))
        fa, fb = random_state(6, 5), random_state(6, 5)
        O.evolve(pa, fa, 0, 12)
        O.evolve(pb, fb, 0, 12)
        assert np.max(np.abs(fa - fb)) < 1e-12
        oa, ob = O.observables(pa, fa, 12), O.observables(pb, fb, 12)
        assert abs(oa["sum_L"] - ob["sum_L"]) < 1e-10 * abs(oa["sum_L"])


def test_minkowski_energy_second_order():
    """With a = 1 the time-centred energy is conserved to O(dt^2): halving dt cuts
    the largest excursion by about 4."""
    out = []
    for dt in (0.05, 0.025):
        p = O.Params(N=8, era=O.MINKOWSKI, dt=dt, seed=13)
        f = random_state(8, 17, phi_amp=0.8, pi_amp=0.3, th_amp=0.3, e_amp=0.2)
        H0 = O.energy(p, f, 0)
        n = int(round(3.0 / dt))
        dev = 0.0
        for q in range(n):
            O.evolve(p, f, q, 1)
            dev = max(dev, abs(O.energy(p, f, q + 1) - H0))
        out.append(dev / H0)
    assert 3.0 < out[0] / out[1] < 5.0, out
    assert out[1] < 2e-2


def test_light_cone_window_locality():
    """After k steps a site depends only on the initial data within Chebyshev
    radius k: a window evolved alone matches the full lattice bit for bit in its
    interior, also across the periodic seam."""
    p = O.Params(N=16, era=O.MATTER, s=1.0, seed=7)
    f = O.init(p)
    k = 3
    O.evolve(p, f, 0, k)
    org = (12, 5, 14)
    w = O.init(p, M=10, origin=org)
    O.evolve(p, w, 0, k)
    idx = [(np.arange(k, 10 - k) + o) % 16 for o in org]
    sub = f[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]
    assert np.array_equal(w[:, k:10 - k, k:10 - k, k:10 - k], sub)


# ---------------------------------------------------------------- diagnostics
@pytest.mark.parametrize("axis,N", [(2, 12), (0, 9), (1, 10)])
def test_straight_string_windings(axis, N):
    """Four straight strings along `axis`: exactly one pierced plaquette per lattice
    spacing per string, windings +-1 summing to zero, none in the other planes;
    unchanged by a random gauge transform."""
    f = straight_strings(N, axis=axis)
    w = O.windings(f)
    plane = {2: 0, 1: 1, 0: 2}[axis]       # xy pierced by z-strings, xz by y, yz by x
    for q in range(3):
        if q == plane:
            assert np.sum(np.abs(w[q])) == 4 * N
            assert np.sum(w[q]) == 0
            per_layer = np.sum(np.abs(w[q]), axis=tuple(d for d in range(3) if d != 2 - axis))
            assert np.all(per_layer == 4)
        else:
            assert not np.any(w[q])
    g = f.copy()
    O.gauge_transform(g, random_angles(N, 3))
    assert np.array_equal(O.windings(g), w)
    p = O.Params(N=N)
    o = O.observables(p, f, 0)
    assert o["sum_abs_W"] == 4 * N and o["n_pierced"] == 4 * N
    assert math.isclose(o["xi_W"], math.sqrt(N ** 3 * p.dx ** 3 / (math.pi / 6 * p.dx * 4 * N)))


def test_bps_string_tension_fixes_xi_L():
    """xi_L = sqrt(-mu / mean L) with mu = 2 pi sigma^2 (Eq. defXiV2; mu is the
    tension of a string at critical coupling lambda0 = 2 e0^2).  A static straight
    Nielsen-Olesen string, its profile solved from the Bogomolny equations with
    scipy (inputs.bps_string), put on lattices of spacing 1/2, 1/4, 1/8 in the same
    16^3 box: its Lagrangian per unit length must tend to -2 pi sigma^2, so that
    xi_L tends to the box side (one string of length N dx in a volume (N dx)^3)
    with an O(dx^2) error -- ratio 4 per halving.  This fixes mu (2 pi, not pi),
    the square root, and the weights of K, |D phi|^2, V, E_el and the magnetic
    term in L together (a halved magnetic coefficient misses by several per cent).
    The string pierces exactly one xy plaquette per lattice spacing."""
    err = []
    for N in (32, 64, 128):
        dx = 16.0 / N
        f = bps_string(N, dx)
        p = O.Params(N=N, dx=dx, dt=dx / 4, era=O.MINKOWSKI, lambda0=2.0, e0=1.0, sigma=1.0)
        o = O.observables(p, f, 0)
        assert o["sum_abs_W"] == N and o["n_pierced"] == N
        assert list(o["sum_abs_W_plane"]) == [N, 0, 0]
        mu_lat = -o["sum_L"] * dx ** 3 / (N * dx)          # tension on the lattice
        assert abs(mu_lat / (2 * math.pi) - 1) < 0.02
        err.append(o["xi_L"] / (N * dx) - 1.0)
    assert 0 < err[2] < 1e-3
    for a, b in zip(err, err[1:]):
        assert 3.6 < a / b < 4.4, err
    assert abs((4 * err[2] - err[1]) / 3) < 2e-5, err       # Richardson: the O(dx^2) term removed


def test_pure_gauge_has_no_winding():
    f = O.new_fields(8)
    f[0] = 1.0
    O.gauge_transform(f, random_angles(8, 8))
    assert not np.any(O.windings(f))


def test_velocity_estimators_closed_forms():
    """Pi = 0 gives R = 0 exactly.  A lattice plane wave phi = r e^{ik.x},
    Pi = i w r e^{ik.x} (w the lattice frequency) has |Pi|^2 = |D phi|^2 at every
    site, so R = 1 and <v^2>_V = <v^2>_L = 1 for any weight; with lambda = 0 plus a
    uniform E it is pure radiation, p = rho / 3 and <v^2>_omega = 1.  A uniform
    field off the vacuum at rest has p = -rho and <v^2>_omega = -1."""
    p = O.Params(N=8, era=O.MINKOWSKI, seed=2)
    f = O.init(p)
    o = O.observables(p, f, 0)
    assert o["v2_V"] == 0.0 and o["R_L"] == 0.0
    N, m, r = 8, (1, 0, 2), 0.5
    i, j, k = coords(N)
    ph = 2 * np.pi * (m[0] * i + m[1] * j + m[2] * k) / N
    w = math.sqrt(4 / p.dx ** 2 * sum(math.sin(math.pi * mj / N) ** 2 for mj in m))
    f = O.new_fields(N)
    f[0], f[1] = r * np.cos(ph), r * np.sin(ph)
    f[2], f[3] = -w * r * np.sin(ph), w * r * np.cos(ph)
    o = O.observables(p, f, 0)
    assert abs(o["R_V"] - 1) < 1e-13 and abs(o["R_L"] - 1) < 1e-13
    assert abs(o["v2_V"] - 1) < 1e-13 and abs(o["v2_L"] - 1) < 1e-13
    p0 = O.Params(N=8, era=O.MINKOWSKI, lambda0=0.0)
    f[7] = 0.3
    o = O.observables(p0, f, 0)
    assert abs(o["v2_omega"] - 1) < 1e-13
    f = O.new_fields(N)
    f[0] = 0.4
    o = O.observables(p, f, 0)
    assert abs(o["v2_omega"] + 1) < 1e-13
    assert o["sum_L"] < 0 and abs(o["sum_L"] + o["sum_rho"]) < 1e-12


def _mode_ode(p, omega2, which, y0, t0, t1):
    """Single lattice mode in an expanding background, from the continuous-time
    equations of the model at linear order:
      scalar (lambda = 0, theta = 0): (a^2 A')' = -a^2 w^2 A
      gauge  (phi = 0):               (A' / e^2)' = -(w^2 / e^2) A
    with e = e0 a^(s-1) (Eq. 7); integrated with scipy's DOP853."""
    from scipy.integrate import solve_ivp
    alpha = {0: 0, 1: 1, 2: 2}[p.era]

    def rhs(t, y):
        a = (t / p.tau_ref) ** alpha
        H = alpha / t
        fric = 2 * H if which == "scalar" else -2 * (p.s - 1) * H
        return [y[1], -fric * y[1] - omega2 * y[0]]

    sol = solve_ivp(rhs, (t0, t1), y0, method="DOP853", rtol=1e-13, atol=1e-16)
    return sol.y[:, -1]


@pytest.mark.parametrize("which", ["scalar", "gauge"])
def test_lattice_mode_second_order_in_expanding_background(which):
    """A small lattice plane wave (scalar) or transverse link wave (gauge) in the
    radiation era with s = 0 must converge at second order in dt to its mode ODE;
    this fixes the time-centring of the Laplacian and curl coefficients."""
    N, m = 8, np.array([1, 2, 1])
    p0 = O.Params(N=N, era=O.RADIATION, s=0.0, lambda0=0.0, tau_ref=2.0, tau0=1.0)
    sn = np.sin(np.pi * m / N)
    omega2 = 4 / p0.dx ** 2 * float(np.sum(sn * sn))
    i, j, k = coords(N)
    ph = 2 * np.pi * (m[0] * i + m[1] * j + m[2] * k) / N
    pol = np.cross(sn, [0.3, -0.7, 0.2])
    pol *= 1e-6 / np.linalg.norm(pol)
    T, y0 = 1.6, [1.0, 0.7]
    ref = _mode_ode(p0, omega2, which, y0, p0.tau0, p0.tau0 + T)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        p = O.Params(**{**p0.__dict__, "dt": dt})
        back = _mode_ode(p, omega2, which, y0, p.tau0, p.tau0 - dt / 2)
        f = O.new_fields(N)
        if which == "scalar":
            f[0], f[2] = 1e-3 * y0[0] * np.cos(ph), 1e-3 * back[1] * np.cos(ph)
        else:
            for d in range(3):
                shape = np.cos(ph + np.pi * m[d] / N)
                f[4 + d], f[7 + d] = pol[d] * y0[0] * shape, pol[d] * back[1] * shape
        n = int(round(T / dt))
        O.evolve(p, f, 0, n)
        if which == "scalar":
            got = f[0, 0, 0, 0] / 1e-3
        else:
            d = int(np.argmax(np.abs(pol)))
            got = f[4 + d, 0, 0, 0] / (pol[d] * np.cos(np.pi * m[d] / N))
        errs.append(abs(got - ref[0]))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


def test_stress_energy_special_cases():
    """Legendre structure of the per-site diagnostics (Eq. 2 and the pressure):
    L = rho for purely kinetic states and L = -rho for states at rest; equations of
    state w = p/rho of 1 (homogeneous kinetic scalar), 1/3 (electric or magnetic
    field alone), -1 (vacuum energy); and for states the kicks leave unchanged the
    diagnostic energy dx^3 sum rho equals the conserved energy."""
    N = 6
    p = O.Params(N=N, era=O.MINKOWSKI, lambda0=0.0)
    i, j, k = coords(N)

    def check(f, w, Lsign, pp=p, static=False):
        o = O.observables(pp, f, 0)
        assert o["sum_rho"] > 0
        assert abs(o["sum_p"] - w * o["sum_rho"]) < 1e-12 * o["sum_rho"]
        assert abs(o["sum_L"] - Lsign * o["sum_rho"]) < 1e-12 * o["sum_rho"]
        if static:
            assert abs(O.energy(pp, f, 0) - o["energy"]) < 1e-12 * o["energy"]

    f = O.new_fields(N); f[2], f[3] = 0.3, -0.4
    check(f, 1.0, +1)                                   # kinetic scalar
    f = O.new_fields(N); f[7], f[8], f[9] = 0.2, -0.1, 0.4
    f[4] = 0.3
    check(f, 1.0 / 3.0, +1, static=True)                # electric field
    f = O.new_fields(N); f[5] = 2 * np.pi * i / N       # uniform flux through xy plaquettes
    check(f, 1.0 / 3.0, -1, static=True)                # magnetic field
    pv = O.Params(N=N, era=O.MINKOWSKI, lambda0=2.0)
    f = O.new_fields(N); f[0] = 0.4
    check(f, -1.0, -1, pp=pv)                           # vacuum energy
    g = random_state(N, 8)
    g[2:4] = 0.0
    g[7:10] = 0.0
    o = O.observables(pv, g, 0)                         # at rest: L = -rho
    assert abs(o["sum_L"] + o["sum_rho"]) < 1e-12 * o["sum_rho"]


# ---------------------------------------------------------------- compact theta
def test_wrapped_theta_is_the_same_evolution_mod_2pi():
    """theta only enters through e^{i theta}: evolving with theta reduced to
    [-pi, pi] after every drift gives the non-compact evolution's phi, Pi, E
    (to rounding) and its theta modulo 2 pi, with every phase inside [-pi, pi].
    A reduction by pi, of the wrong component, or with the wrong sign breaks it."""
    N = 6
    f = random_state(N, 31, th_amp=9.0, e_amp=2.0)      # phases far outside [-pi, pi]
    a = O.Params(N=N, era=O.MINKOWSKI, seed=1)
    b = O.Params(N=N, era=O.MINKOWSKI, seed=1, wrap_theta=True)
    fa, fb = f.copy(), f.copy()
    O.evolve(a, fa, 0, 25)
    O.evolve(b, fb, 0, 25)
    assert np.max(np.abs(fb[4:7])) <= np.pi * (1 + 1e-15)
    assert np.max(np.abs(fa[4:7])) > 3 * np.pi
    for c in (0, 1, 2, 3, 7, 8, 9):
        assert np.max(np.abs(fa[c] - fb[c])) <= 1e-11 * max(1.0, np.max(np.abs(fa[c]))), c
    d = np.remainder(fa[4:7] - fb[4:7] + np.pi, 2 * np.pi) - np.pi
    assert np.max(np.abs(d)) < 1e-11
    # every other observable agrees; max |theta| is the one that changes
    oa, ob = O.observables(a, fa, 25), O.observables(b, fb, 25)
    for k in ("sum_L", "sum_rho", "sum_p", "sum_B", "sum_gauss2"):
        assert abs(oa[k] - ob[k]) <= 1e-10 * max(1.0, abs(oa[k])), k
    assert oa["sum_abs_W"] == ob["sum_abs_W"]
    assert ob["max_abs_theta"] <= np.pi * (1 + 1e-15) < oa["max_abs_theta"]
    # phases already inside [-pi, pi] are left bit for bit as they are
    g = random_state(N, 32, th_amp=0.5, e_amp=0.05)
    ga, gb = g.copy(), g.copy()
    O.evolve(a, ga, 0, 3)
    O.evolve(b, gb, 0, 3)
    assert np.array_equal(ga, gb)


# ---------------------------------------------------------------- core growth
def test_core_growth_is_two_runs_joined_at_tau_ref():
    """Core growth (Sec. 2): exponent s before tau_ref, 1 after.  With tau_ref on a
    half step, the schedule is exactly an s run up to the step whose upper half
    time is tau_ref followed by an s = 1 run (a(tau_ref) = 1 gives both branches
    e0 and lambda0 at the switch), and it differs from either run alone."""
    N, k, n = 8, 8, 16
    kw = dict(N=N, era=O.RADIATION, dt=0.125, tau0=1.0, tau_ref=1.0 + 7.5 * 0.125, seed=12)
    f0 = O.init(O.Params(s=-1.0, **kw))
    f0[2:] = random_state(N, 33, pi_amp=0.2, th_amp=0.3, e_amp=0.2)[2:]
    cg = O.evolve(O.Params(s=-1.0, core_growth=True, **kw), f0.copy(), 0, n)
    joined = O.evolve(O.Params(s=-1.0, **kw), f0.copy(), 0, k)
    O.evolve(O.Params(s=1.0, **kw), joined, k, n - k)
    assert np.array_equal(cg, joined)
    only_s = O.evolve(O.Params(s=-1.0, **kw), f0.copy(), 0, n)
    only_1 = O.evolve(O.Params(s=1.0, **kw), f0.copy(), 0, n)
    assert np.max(np.abs(cg - only_s)) > 1e-4 and np.max(np.abs(cg - only_1)) > 1e-4
    # s = 1 throughout is the true equations, whatever the switch time
    a = O.evolve(O.Params(s=1.0, core_growth=True, **kw), f0.copy(), 0, n)
    assert np.array_equal(a, only_1)
