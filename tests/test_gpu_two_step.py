"""Two leapfrog steps per pass (AH_FLAG_TWO_STEP, k_fused2) on the GPU.

The two-step kernel evaluates each step with the single-step kernel's
formulas (the compiler may fuse a multiply-add differently, so the two agree
to FP32 rounding, not bit for bit); after 20 steps both equal the FP64
oracle within the FP32 parity bar (1e-5 of each component's scale), and each
other within the same bar after any mix of step counts.  Lattices span several
tiles of the kernel (30 x 6 written sites per CTA for the 32 x 8 shapes) with
ragged edges, several z chunks, and the periodic seams.
"""
import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah
from inputs import random_state

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TWO = ah.AH_FLAG_TWO_STEP


def rel_err(got, ref, theta_mod_2pi=False):
    """Per-component max |got - ref| / max(max |ref|, 1); with theta_mod_2pi the
    link phases are compared modulo 2 pi (in units of pi)."""
    out = []
    for c in range(10):
        d = got[c] - ref[c]
        if theta_mod_2pi and 4 <= c <= 6:
            out.append(float(np.max(np.abs(np.remainder(d + np.pi, 2 * np.pi) - np.pi)) / np.pi))
        else:
            out.append(float(np.max(np.abs(d)) / max(np.max(np.abs(ref[c])), 1.0)))
    return out


def n_shapes():
    with ah.Sim(8, flags=TWO) as g:
        return g.info["n_variants"]


def run(N, f, nsteps, flags, era, s, variant=None, step0=3, chunks=None, **kw):
    """Fields after `nsteps` steps (ah_step called with the counts in `chunks`
    when given) from the FP32-rounded state f set at step `step0`."""
    with ah.Sim(N, era=era, s=s, seed=1, flags=flags, **kw) as g:
        if variant is not None:
            g.set_variant(variant)
        g.set_fields(f, step=step0)
        f0 = g.fields()
        for n in (chunks or [nsteps]):
            g.step(n)
        assert g.n == step0 + nsteps
        return f0, g.fields(), g.observables()


# (N, era, s): the smallest lattice, one tile, ragged tiles in x and y, several
# z chunks (N = 64, 70: 16- and 18-plane chunks), all three eras
CASES = [(4, ah.AH_MINKOWSKI, 0.0), (6, ah.AH_MATTER, 1.0), (17, ah.AH_RADIATION, -0.5),
         (33, ah.AH_RADIATION, 0.0), (40, ah.AH_MATTER, 1.0), (64, ah.AH_RADIATION, 0.0),
         (70, ah.AH_MATTER, 0.5)]


@pytest.mark.parametrize("N,era,s", CASES)
def test_two_step_equals_single_steps(N, era, s):
    """21 steps (ten passes and one single step) against 21 single fused steps."""
    f = random_state(N, N + 11)
    _, one, o1 = run(N, f, 21, 0, era, s, tau_ref=9.0)
    _, two, o2 = run(N, f, 21, TWO, era, s, tau_ref=9.0)
    assert max(rel_err(two, one)) <= TOL32, rel_err(two, one)
    assert o2["step"] == o1["step"] and o2["nonfinite"] == 0
    for k in range(8):
        assert abs(o2["sums"][k] - o1["sums"][k]) <= 1e-5 * abs(o1["sums"][1]), k


@pytest.mark.parametrize("N,era,s", CASES)
def test_every_two_step_shape_matches_oracle(N, era, s):
    f = random_state(N, N + 5)
    p = O.Params(N=N, era=era, s=s, seed=1, tau_ref=9.0)
    ref = None
    for v in range(n_shapes()):
        f0, got, _ = run(N, f, 20, TWO, era, s, variant=v, tau_ref=9.0)
        if ref is None:
            ref = O.evolve(p, f0.copy(), 3, 20)
        assert max(rel_err(got, ref)) <= TOL32, (v, rel_err(got, ref))


def test_odd_and_mixed_step_counts():
    """Calls of 1, 3, 2, 5 and 0 steps (pairs plus single steps in between) give
    the fields of 11 single steps."""
    N = 36
    f = random_state(N, 8)
    _, one, _ = run(N, f, 11, 0, ah.AH_RADIATION, 0.0, tau_ref=9.0)
    _, two, _ = run(N, f, 11, TWO, ah.AH_RADIATION, 0.0, chunks=[1, 3, 2, 5, 0], tau_ref=9.0)
    assert max(rel_err(two, one)) <= TOL32, rel_err(two, one)


def test_wrap_and_core_growth_in_two_step_mode():
    """Compact phases (reduced after each of the two drifts) and the core-growth
    schedule switching between the two steps of a pass."""
    N = 30
    f = random_state(N, 21, th_amp=9.0)
    flags = ah.AH_FLAG_WRAP_THETA | ah.AH_FLAG_CORE_GROWTH
    kw = dict(tau_ref=2.05, tau0=1.0, dt=0.1)          # tau crosses tau_ref inside a pair
    _, one, _ = run(N, f, 20, flags, ah.AH_RADIATION, -1.0, step0=0, **kw)
    _, two, _ = run(N, f, 20, flags | TWO, ah.AH_RADIATION, -1.0, step0=0, **kw)
    assert max(rel_err(two, one, theta_mod_2pi=True)) <= TOL32, rel_err(two, one, theta_mod_2pi=True)
    assert np.max(np.abs(two[4:7])) <= np.pi * (1 + 1e-6)


def test_two_step_info_autotune_and_state_size():
    N = 64
    with ah.Sim(N, seed=4, flags=TWO | ah.AH_FLAG_AUTOTUNE) as g:
        info = g.info
        assert info["variant_name"].startswith("two_") and 0 <= info["variant"] < info["n_variants"]
        assert info["state_bytes"] == 20 * ((N ** 3 + 63) // 64 * 64) * 4
        with pytest.raises(ah.AhError):
            g.set_variant(info["n_variants"])
        start = g.fields()                   # autotune restored the initial state
    with ah.Sim(N, seed=4) as g:
        assert np.array_equal(start, g.fields())


def test_1024cubed_two_step_light_cone_windows():
    """1024^3 FP32, matter era, s = 1, seed 3 (the bench lattice) in two-step mode,
    autotuned shape: after 20 steps (10 passes) three 16^3 windows, two across
    the periodic seam, equal the oracle's evolution of (16 + 2*20)^3 windows; the
    Gauss residual stays at FP32 roundoff over the whole lattice."""
    N, k, b = 1024, 20, 16
    p = O.Params(N=N, era=ah.AH_MATTER, s=1.0, seed=3)
    with ah.Sim(N, era=ah.AH_MATTER, s=1.0, seed=3, flags=TWO | ah.AH_FLAG_AUTOTUNE) as g:
        g.step(k)
        for org in [(1016, 5, 1019), (300, 1010, 7), (511, 512, 640)]:
            M = b + 2 * k
            win = O.init(p, M=M, origin=[(o - k) % N for o in org])
            win32 = win.astype(np.float32).astype(np.float64)
            O.evolve(p, win32, 0, k)
            got = g.fields(*org, b, b, b)
            assert max(rel_err(got, win32[:, k:k + b, k:k + b, k:k + b])) <= TOL32, org
        o = g.observables()
    assert o["n_sites"] == N ** 3 and o["nonfinite"] == 0 and o["gauss_rel"] < 1e-5


def test_1024cubed_weak_field_kernel_light_cone_windows():
    """The launches the bench times: the 1024^3 bench lattice in two-step mode
    after whole-lattice observables at step 0 (max |theta| = 0), so all ten
    passes of 20 steps run the kernel for weak gauge fields; three 16^3
    windows, two across the periodic seam, equal the oracle's evolution of
    (16 + 2*20)^3 windows."""
    N, k, b = 1024, 20, 16
    p = O.Params(N=N, era=ah.AH_MATTER, s=1.0, seed=3)
    with ah.Sim(N, era=ah.AH_MATTER, s=1.0, seed=3, flags=TWO) as g:
        assert g.observables()["max_abs_theta"] <= 2.0 ** -7
        g.step(k)
        assert g.info["weak_field_launches"] == k // 2
        for org in [(1020, 1013, 2), (77, 1015, 1009), (640, 333, 511)]:
            M = b + 2 * k
            win = O.init(p, M=M, origin=[(o - k) % N for o in org])
            win32 = win.astype(np.float32).astype(np.float64)
            O.evolve(p, win32, 0, k)
            got = g.fields(*org, b, b, b)
            assert max(rel_err(got, win32[:, k:k + b, k:k + b, k:k + b])) <= TOL32, org
        o = g.observables()
    assert o["nonfinite"] == 0 and o["gauss_rel"] < 1e-5


def test_1300cubed_two_step_64bit_site_indices():
    """N^3 >= 2^31 takes the 64-bit-index instantiation: 1300^3 FP32 in two-step
    mode (20 arrays, 176 GB); windows beyond linear index 2^31 and across the
    seam equal the oracle after 20 steps."""
    N, k, b = 1300, 20, 12
    assert N ** 3 >= 2 ** 31
    p = O.Params(N=N, era=ah.AH_RADIATION, s=0.0, seed=6)
    with ah.Sim(N, era=ah.AH_RADIATION, s=0.0, seed=6, flags=TWO) as g:
        g.step(k)
        for org in [(1295, 3, 1290), (640, 1297, 1280)]:
            M = b + 2 * k
            win = O.init(p, M=M, origin=[(o - k) % N for o in org])
            win32 = win.astype(np.float32).astype(np.float64)
            O.evolve(p, win32, 0, k)
            got = g.fields(*org, b, b, b)
            assert max(rel_err(got, win32[:, k:k + b, k:k + b, k:k + b])) <= TOL32, org


@pytest.mark.parametrize("th_amp,e_amp", [(2e-4, 1e-4), (7e-3, 0.3)])
def test_weak_field_kernel_matches_oracle(th_amp, e_amp):
    """After whole-lattice observables with max |theta| <= 2^-7 the pairs run
    the kernel specialised to weak gauge fields: (a) phases that stay tiny, so
    every warp takes the two-term sine/cosine forms; (b) phases just below
    2^-7 that the electric field drives past 2^-6 within a step, so warps fall
    back to the polynomials.  Both equal the oracle and the general two-step
    kernel after 20 steps."""
    N = 40
    f = random_state(N, 61, th_amp=th_amp, e_amp=e_amp)
    p = O.Params(N=N, era=ah.AH_MATTER, s=1.0, seed=1, tau_ref=9.0)
    with ah.Sim(N, era=ah.AH_MATTER, s=1.0, seed=1, flags=TWO, tau_ref=9.0) as g:
        g.set_fields(f, step=3)
        f0 = g.fields()
        assert g.observables()["max_abs_theta"] <= 2.0 ** -7
        g.step(20)
        got = g.fields()
        assert g.info["weak_field_launches"] == 10
    _, general, _ = run(N, f, 20, TWO, ah.AH_MATTER, 1.0, tau_ref=9.0)   # no observables first: general kernel
    ref = O.evolve(p, f0.copy(), 3, 20)
    assert max(rel_err(got, ref)) <= TOL32, rel_err(got, ref)
    assert max(rel_err(got, general)) <= TOL32, rel_err(got, general)


def test_strong_fields_and_new_fields_keep_the_general_kernel():
    """Phases beyond 2^-7 at the last observables, or fields set since, keep
    the general two-step kernel."""
    N = 24
    with ah.Sim(N, flags=TWO) as g:
        g.set_fields(random_state(N, 62, th_amp=0.4), 0)
        g.observables()
        g.step(4)
        assert g.info["weak_field_launches"] == 0
        g.set_fields(random_state(N, 63, th_amp=1e-4), 4)
        assert g.observables()["max_abs_theta"] <= 2.0 ** -7
        g.step(2)
        assert g.info["weak_field_launches"] == 1
        g.set_fields(random_state(N, 63, th_amp=1e-4), 6)
        g.step(2)
        assert g.info["weak_field_launches"] == 1
