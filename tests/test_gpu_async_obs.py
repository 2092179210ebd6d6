"""Asynchronous observables (ah_observables_start / ah_observables_finish, GPU).

The pass reads the state at the start (the snapshot) on a second stream while
later steps go on; a launch that would overwrite the snapshot waits for it.  The
result must be that of ah_observables on the same state, and the evolution must
be exactly the one without the pass.  (A two-step simulation may hand the pass
to its next two-step launch instead; it does so here only when asked to, or on
states with few pierced plaquettes: test_gpu_fused_diag.py.)"""
import numpy as np
import pytest

import paper_1809_00995_gb300 as ah
from inputs import random_state

pytestmark = pytest.mark.gpu


def same_obs(a, b):
    assert a["step"] == b["step"] and a["tau"] == b["tau"]
    assert a["sums"] == b["sums"]
    assert a["wind_abs_plane"] == b["wind_abs_plane"] and a["wind_plane"] == b["wind_plane"]
    assert a["n_pierced"] == b["n_pierced"] and a["gauss_max"] == b["gauss_max"]


@pytest.mark.parametrize("precision,flags,later", [(ah.AH_FP32, ah.AH_FLAG_TWO_STEP, 7), (ah.AH_FP32, 0, 5),
                                                   (ah.AH_FP64, 0, 4), (ah.AH_FP32, ah.AH_FLAG_TWO_STEP, 1)])
def test_async_observables_equal_sync_and_leave_the_evolution_alone(precision, flags, later):
    N = 40
    kw = dict(precision=precision, kernel=ah.AH_KERNEL_FUSED, era=ah.AH_MATTER, s=1.0, seed=17, flags=flags)
    with ah.Sim(N, **kw) as a, ah.Sim(N, **kw) as b:
        a.step(24)
        ref = a.observables()
        a.step(later)
        b.step(24)
        b.observables_start()
        b.step(later)                       # overlaps the pass (the first two-step launch) or waits for it
        got = b.observables_finish()
        same_obs(got, ref)
        assert np.array_equal(a.fields(), b.fields())
        # a second round on the same simulation
        b.observables_start()
        b.step(2)
        got2 = b.observables_finish()
        ref2 = a.observables()
        same_obs(got2, ref2)


def test_async_observables_busy_and_argument_rules():
    with ah.Sim(16, precision=ah.AH_FP32, flags=ah.AH_FLAG_TWO_STEP) as g:
        with pytest.raises(ah.AhError) as e:
            g.observables_finish()
        assert e.value.status == ah.AH_ERR_ARG
        g.observables_start()
        for call in (g.observables_start, g.observables):
            with pytest.raises(ah.AhError) as e:
                call()
            assert e.value.status == ah.AH_ERR_BUSY
        g.step(4)
        o = g.observables_finish()
        assert o["step"] == 0
        assert g.observables()["step"] == 4


def test_async_observables_settle_a_list_overflow_on_the_device():
    """A 128^3 state of real +-1 fields and theta = 0 puts about 7/8 of its 6.3e6
    plaquettes on the branch cut, more than the simulation's list holds (2^20):
    the asynchronous pass recounts every winding in FP64 on the device, and its
    counts equal those of the synchronous path (which recounts on the host's
    decision); the energies agree to the FP32 diagnostic tolerance."""
    N = 128
    f = random_state(N, 5)
    rng = np.random.Generator(np.random.PCG64(6))
    f[0] = rng.choice([-1.0, 1.0], size=(N, N, N))
    f[1] = 0.0
    f[4:7] = 0.0
    with ah.Sim(N, precision=ah.AH_FP32, seed=5) as g:
        g.set_fields(f, 3)
        ref = g.observables()
        g.observables_start()
        got = g.observables_finish()
    assert got["n_pierced"] > 0
    assert got["wind_abs_plane"] == ref["wind_abs_plane"] and got["wind_plane"] == ref["wind_plane"]
    assert got["n_pierced"] == ref["n_pierced"]
    scale = abs(ref["sums"][1])
    for k in range(8):
        assert abs(got["sums"][k] - ref["sums"][k]) <= 1e-5 * abs(ref["sums"][k]) + 2e-6 * scale, k
