"""Diagnostics folded into the two-step pass (k_fused2_diag, GPU).

An FP32 simulation stepped two steps per launch may defer ah_observables_start
(always with AH_FLAG_FUSED_DIAG; without it when its last observables found
few pierced plaquettes): the next two-step launch reads the state n for its
first step anyway, so it also takes the whole-lattice diagnostics of that
state (Sec. 2: energy sums, Gauss residual, windings of Eq. 9) on the sites it
writes.  The results must be those of the separate pass (ah_observables) on
the same state -- windings, max |G| and max |theta| exactly, sums to the
rounding of a different summation order -- and those of the FP64 oracle
within the FP32 diagnostic tolerances; the evolution must be the one without
diagnostics, bit for bit."""
import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah
from inputs import random_state, straight_strings
from test_gpu_parity import compare_obs, oparams

pytestmark = pytest.mark.gpu

TWO = ah.AH_FLAG_TWO_STEP
FUSED = ah.AH_FLAG_TWO_STEP | ah.AH_FLAG_FUSED_DIAG


def close_obs(got, ref, rel=2e-6):
    """The same per-site FP32 terms summed in another order: each thread's
    compensated partial is within about 2^-23 of its value, so two groupings
    differ by at most a few 1e-7 of sum rho (first-order sums, |L|, |p| <= rho per
    site), of (sum rho)^2 / n_sites (products) or of the Gauss sums themselves."""
    assert got["step"] == ref["step"] and got["tau"] == ref["tau"]
    assert got["wind_abs_plane"] == ref["wind_abs_plane"] and got["wind_plane"] == ref["wind_plane"]
    assert got["n_pierced"] == ref["n_pierced"] and got["nonfinite"] == ref["nonfinite"] == 0
    assert got["gauss_max"] == ref["gauss_max"] and got["max_abs_theta"] == ref["max_abs_theta"]
    s1 = abs(ref["sums"][1])
    s2 = s1 * s1 / ref["n_sites"]
    for k in range(16):
        scale = s1 if k < 8 else (s2 if k < 14 else abs(ref["sums"][k]))
        assert abs(got["sums"][k] - ref["sums"][k]) <= rel * scale, (k, got["sums"][k], ref["sums"][k])


def twin(N, **kw):
    args = dict(precision=ah.AH_FP32, kernel=ah.AH_KERNEL_FUSED, era=ah.AH_MATTER, s=1.0, seed=23, flags=FUSED)
    args.update(kw)
    return ah.Sim(N, **args), ah.Sim(N, **args)


@pytest.mark.parametrize("N", [8, 20, 37, 64])
def test_fused_diagnostics_equal_the_separate_pass_and_the_oracle(N):
    """Ragged tiles (30 x 6 written sites per CTA) and several z chunks; the
    state after 16 steps of the random-phase start has non-zero Pi, E and
    plaquettes near the branch cut."""
    a, b = twin(N)
    with a, b:
        a.step(16)
        snap = a.fields()
        ref = a.observables()
        a.step(6)
        b.step(16)
        b.observables_start()
        b.step(6)                     # the first of three two-step launches takes the diagnostics
        got = b.observables_finish()
        assert b.info["fused_diag_passes"] == 1
        close_obs(got, ref)
        np.testing.assert_array_equal(b.fields(), a.fields())
    compare_obs(got, O.observables(oparams(N, era=ah.AH_MATTER, s=1.0, seed=23), snap, 16), ah.AH_FP32)


@pytest.mark.parametrize("kind", ["random", "large_theta", "real_fields", "strings", "tiny_phi"])
def test_fused_windings_bit_exact_on_hard_snapshots(kind):
    """Snapshots with many plaquettes at or near a branch cut (the near-cut list
    and its FP64 fix-up on the state the pass leaves in place), smooth regions
    where a CTA skips the carries (strings), and edge products that need the
    power-of-two scaling (|phi| ~ 1e-5)."""
    N = 24
    if kind == "random":
        f = random_state(N, 41, phi_amp=1.0, th_amp=3.0)
    elif kind == "large_theta":
        f = random_state(N, 42, th_amp=40.0)
    elif kind == "real_fields":
        f = random_state(N, 43)
        f[1] = 0.0
        f[4:7] = 0.0
    elif kind == "strings":
        f = straight_strings(N, axis=2, x0=0.5, y0=0.25)
    else:
        f = random_state(N, 44, th_amp=2.0)
        f[0:2] *= 1e-5
    with ah.Sim(N, precision=ah.AH_FP32, flags=FUSED) as g:
        g.set_fields(f, 4)
        snap = g.fields()
        ref = g.observables()
        g.observables_start()
        g.step(2)
        got = g.observables_finish()
    close_obs(got, ref)
    oo = O.observables(oparams(N), snap, 4)
    assert list(got["wind_abs_plane"]) == list(oo["sum_abs_W_plane"])
    assert list(got["wind_plane"]) == list(oo["sum_W_plane"])
    assert got["n_pierced"] == oo["n_pierced"]
    if kind == "strings":
        assert got["wind_abs_plane"] == [4 * N, 0, 0]


def test_fused_diagnostics_settle_a_list_overflow():
    """A 128^3 state of real +-1 fields with zero links puts about 5.5e6
    plaquettes on the branch cut, more than the list holds (2^20): the FP64
    recount of the windings runs on the device after the fused launch, on the
    state n.  (The synchronous pass decides on the host and redoes everything
    in FP64, so its energies and max |G| are the exact path's.)"""
    N = 128
    f = random_state(N, 5)
    rng = np.random.Generator(np.random.PCG64(6))
    f[0] = rng.choice([-1.0, 1.0], size=(N, N, N))
    f[1] = 0.0
    f[4:7] = 0.0
    with ah.Sim(N, precision=ah.AH_FP32, seed=5, flags=FUSED) as g:
        g.set_fields(f, 3)
        ref = g.observables()
        g.observables_start()
        g.step(2)
        got = g.observables_finish()
    assert got["n_pierced"] > 0
    assert got["wind_abs_plane"] == ref["wind_abs_plane"] and got["wind_plane"] == ref["wind_plane"]
    assert got["n_pierced"] == ref["n_pierced"]
    assert abs(got["gauss_max"] - ref["gauss_max"]) <= 1e-12 * ref["gauss_max"]
    scale = abs(ref["sums"][1])
    for k in range(8):
        assert abs(got["sums"][k] - ref["sums"][k]) <= 1e-5 * abs(ref["sums"][k]) + 2e-6 * scale, k


def test_deferred_pass_runs_alone_when_no_two_step_launch_takes_it():
    """Without a two-step launch to ride on (finish right away, an odd single
    step, new fields) the pass runs on its own from the state at the start."""
    N = 20
    with ah.Sim(N, precision=ah.AH_FP32, era=ah.AH_RADIATION, seed=9, flags=FUSED) as g:
        g.step(10)
        ref = g.observables()
        g.observables_start()
        got = g.observables_finish()            # nothing stepped
        assert got == ref
        g.observables_start()
        g.step(1)                               # one step: a single-step launch, which the pass precedes
        assert g.observables_finish() == ref
        ref11 = g.observables()
        g.observables_start()
        f = g.fields()
        g.set_fields(f, 11)                     # new fields: the pass reads the state before them
        assert g.observables_finish() == ref11
        assert g.info["fused_diag_passes"] == 0
        g.observables_start()
        g.step(3)                               # one two-step launch takes it, then a single step
        close_obs(g.observables_finish(), ref11)
        assert g.info["fused_diag_passes"] == 1


def test_two_step_simulation_chooses_the_fused_launch_on_smooth_fields():
    """Without the flag: a rough random-phase state (many pierced plaquettes)
    keeps the separate pass, bit for bit that of ah_observables; a smooth state
    with four straight strings (4 N of 3 N^3 plaquettes pierced) hands the next
    pass to the two-step launch."""
    N = 64
    with ah.Sim(N, precision=ah.AH_FP32, era=ah.AH_RADIATION, seed=4, flags=TWO) as g:
        g.step(6)
        ref = g.observables()
        assert ref["n_pierced"] > 1e-3 * 3 * N ** 3
        g.observables_start()
        g.step(2)
        assert g.observables_finish() == ref
        assert g.info["fused_diag_passes"] == 0
        g.set_fields(straight_strings(N, axis=1, x0=0.5, y0=0.25), 8)
        ref = g.observables()
        assert ref["wind_abs_plane"] == [0, 4 * N, 0]
        g.observables_start()
        g.step(2)
        close_obs(g.observables_finish(), ref)
        assert g.info["fused_diag_passes"] == 1
