"""The core-growth schedule (AH_FLAG_CORE_GROWTH) on the GPU against the oracle's
reading of it: exponent s of Eq. 7 before tau_ref, 1 from tau_ref on, every
coupling of a step at its own time."""
import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah

pytestmark = pytest.mark.gpu

TOL = {ah.AH_FP64: 1e-12, ah.AH_FP32: 1e-5}
# tau_ref = 1.93 lies inside step 9 (tau_9 = 1.9, tau_9 + dt/2 = 1.95): that step
# mixes the two exponents, the steps before use s, the steps after use 1
KW = dict(era=ah.AH_RADIATION, s=-1.0, tau0=1.0, tau_ref=1.93, seed=8)


def rel_err(got, ref):
    return [float(np.max(np.abs(got[c] - ref[c])) / max(np.max(np.abs(ref[c])), 1.0)) for c in range(10)]


@pytest.mark.parametrize("kernel", [ah.AH_KERNEL_PLAIN, ah.AH_KERNEL_FUSED])
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_core_growth_matches_oracle(precision, kernel):
    N = 24
    with ah.Sim(N, precision=precision, kernel=kernel, flags=ah.AH_FLAG_CORE_GROWTH, **KW) as g:
        f0 = g.fields()
        g.step(20)
        got = g.fields()
        obs = g.observables()
    p = O.Params(N=N, core_growth=True, **KW)
    ref = O.evolve(p, f0.copy(), 0, 20)
    assert max(rel_err(got, ref)) <= TOL[precision]
    oo = O.observables(p, ref, 20)
    assert abs(obs["sums"][1] - oo["sum_rho"]) <= (1e-10 if precision == ah.AH_FP64 else 1e-5) * abs(oo["sum_rho"])
    # the schedule changes the run
    with ah.Sim(N, precision=precision, kernel=kernel, **KW) as h:
        h.step(20)
        assert max(rel_err(h.fields(), got)) > 1e-4


def test_core_growth_in_a_batch():
    """The batched path takes the same per-step coefficients."""
    cfgs = [ah.config(N, flags=ah.AH_FLAG_CORE_GROWTH, diag_every=0, **KW) for N in (16, 20)]
    cfgs.append(ah.config(12, **KW))
    series, _ = ah.ah_batch_run(cfgs)
    for cfg, ser in zip(cfgs[:2], series[:2]):
        p = O.Params(N=cfg.N, core_growth=True, **KW)
        f = O.init(p).astype(np.float32).astype(np.float64)
        nsteps = int(round((cfg.tau_end - cfg.tau0) / cfg.dt))
        O.evolve(p, f, 0, nsteps)
        oo = O.observables(p, f, nsteps)
        go = series[cfgs.index(cfg)][-1]
        for k, name in enumerate(["sum_L", "sum_rho", "sum_p", "sum_K", "sum_G2", "sum_V", "sum_Eel", "sum_B"]):
            assert abs(go["sums"][k] - oo[name]) <= 1e-4 * abs(oo["sum_rho"]), name


def test_core_growth_stability_is_checked_on_both_stretches():
    """s = 0 in radiation is stable at any a; switching to s = 1 at tau_ref = 1
    makes the stiff mode grow with a = tau up to tau_end = 64 and is refused."""
    kw = dict(era=ah.AH_RADIATION, s=0.0, tau0=1.0, tau_ref=1.0)
    ah.ah_destroy(ah.ah_create_ex(ah.config(256, **kw)))
    with pytest.raises(ah.AhError) as e:
        ah.ah_create_ex(ah.config(256, flags=ah.AH_FLAG_CORE_GROWTH, **kw))
    assert e.value.status == ah.AH_ERR_UNSTABLE
