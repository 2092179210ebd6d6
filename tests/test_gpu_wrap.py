"""Compact link phases (AH_FLAG_WRAP_THETA) on the GPU against the oracle's
compact reading, and the FP32 accuracy it buys when theta has drifted far
from zero.

theta is compared modulo 2 pi (a phase within one rounding of +-pi may be
reduced on one side and not on the other); every other component as in the
parity tests.
"""
import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah
from inputs import random_state

pytestmark = pytest.mark.gpu

TOL = {ah.AH_FP64: 1e-12, ah.AH_FP32: 1e-5}


def errors_mod_2pi(got, ref):
    """Per-component max error scaled as in the parity tests; theta mod 2 pi."""
    out = []
    for c in range(10):
        d = got[c] - ref[c]
        if 4 <= c <= 6:
            d = np.remainder(d + np.pi, 2 * np.pi) - np.pi
            out.append(float(np.max(np.abs(d)) / np.pi))
        else:
            out.append(float(np.max(np.abs(d)) / max(np.max(np.abs(ref[c])), 1.0)))
    return out


def run(N, precision, kernel, f, nsteps, wrap, variant=None, era=ah.AH_MINKOWSKI):
    flags = ah.AH_FLAG_WRAP_THETA if wrap else 0
    with ah.Sim(N, precision=precision, kernel=kernel, era=era, seed=1, flags=flags) as g:
        if variant is not None:
            g.set_variant(variant)
        g.set_fields(f, step=0)
        f0 = g.fields()
        g.step(nsteps)
        return f0, g.fields(), g.observables()


@pytest.mark.parametrize("kernel", [ah.AH_KERNEL_PLAIN, ah.AH_KERNEL_FUSED])
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_wrapped_fields_match_oracle(precision, kernel):
    """FP64: the compact oracle to rounding.  FP32: phases near 9 carry absolute
    rounding errors 30 times those of the parity tests' states, which the
    nonlinear kicks then amplify, so the FP32 bar is the same run without the
    reduction against the non-compact oracle: the reduction may not be less
    accurate than that (and both stay below 2e-4)."""
    N = 20
    f = random_state(N, 41, th_amp=9.0)          # most phases outside [-pi, pi]
    f0, got, obs = run(N, precision, kernel, f, 20, wrap=True)
    ref = O.evolve(O.Params(N=N, era=O.MINKOWSKI, seed=1, wrap_theta=True), f0.copy(), 0, 20)
    err = max(errors_mod_2pi(got, ref))
    if precision == ah.AH_FP64:
        assert err <= TOL[precision]
    else:
        g0, plain, _ = run(N, precision, kernel, f, 20, wrap=False)
        assert np.array_equal(g0, f0)
        ref_nw = O.evolve(O.Params(N=N, era=O.MINKOWSKI, seed=1), f0.copy(), 0, 20)
        err_nw = max(errors_mod_2pi(plain, ref_nw))
        assert err <= max(TOL[precision], 1.5 * err_nw) and err < 2e-4, (err, err_nw)
    assert np.max(np.abs(got[4:7])) <= np.pi * (1 + 1e-6)
    assert obs["max_abs_theta"] <= np.pi * (1 + 1e-6)


@pytest.mark.parametrize("N", [37, 64])
def test_every_step_shape_wraps(N):
    """Each compile-time shape of every step kernel family applies the reduction."""
    f = random_state(N, 42, th_amp=9.0)
    p = O.Params(N=N, era=O.MINKOWSKI, seed=1, wrap_theta=True)
    ref = None
    for v in range(ah.ah_variant_count(ah.AH_FP32)):
        try:
            f0, got, _ = run(N, ah.AH_FP32, ah.AH_KERNEL_FUSED, f, 6, wrap=True, variant=v)
        except ah.AhError as e:
            assert e.status == ah.AH_ERR_ARG and N % 32 != 0
            continue
        if ref is None:
            ref = O.evolve(p, f0.copy(), 0, 6)
        assert max(errors_mod_2pi(got, ref)) <= TOL[ah.AH_FP32], v
        assert np.max(np.abs(got[4:7])) <= np.pi * (1 + 1e-6), v


def test_wrapping_keeps_fp32_resolution_at_large_theta():
    """An FP32 state whose phases sit near 14 pi (a physically identical copy of a
    state near 0) rounds every theta update at ulp(44) = 4e-6 without the
    reduction; with it the FP32 run tracks the FP64 oracle more closely."""
    N = 24
    f = random_state(N, 43, th_amp=0.5, e_amp=0.05, pi_amp=0.05)
    f[4:7] += 14 * np.pi
    f = f.astype(np.float32).astype(np.float64)           # exactly representable start
    p = O.Params(N=N, era=O.MINKOWSKI, seed=1)
    f0a, nowrap, _ = run(N, ah.AH_FP32, ah.AH_KERNEL_FUSED, f, 400, wrap=False)
    f0b, wrap, _ = run(N, ah.AH_FP32, ah.AH_KERNEL_FUSED, f, 400, wrap=True)
    assert np.array_equal(f0a, f) and np.array_equal(f0b, f)
    ref = O.evolve(p, f.copy(), 0, 400)
    ea, eb = errors_mod_2pi(nowrap, ref), errors_mod_2pi(wrap, ref)
    # the reduced run rounds once at |theta| ~ 44 (its first drift), the other at
    # every step: theta and the fields it drives are several times closer
    assert max(eb[4:7]) * 3 < max(ea[4:7]), (ea, eb)
    assert max(eb) * 2 < max(ea), (ea, eb)


def test_batched_path_wraps_theta():
    """A batched lattice with AH_FLAG_WRAP_THETA gives the single-lattice run's
    observables (same flag) within the FP32 diagnostic tolerance, with every
    phase in [-pi, pi] (max |theta| reported by the final diagnostics)."""
    kw = dict(era=ah.AH_MINKOWSKI, seed=7, flags=ah.AH_FLAG_WRAP_THETA, diag_every=0, tau_end=31.0)
    cfgs = [ah.config(24, **kw), ah.config(16, **kw)]
    series, _ = ah.ah_batch_run(cfgs)
    for cfg, ser in zip(cfgs, series):
        with ah.Sim(cfg.N, era=ah.AH_MINKOWSKI, seed=7, flags=ah.AH_FLAG_WRAP_THETA, tau_end=31.0,
                    kernel=ah.AH_KERNEL_FUSED) as g:
            g.step(int(round((cfg.tau_end - cfg.tau0) / cfg.dt)))
            ref = g.observables()
        got = ser[-1]
        assert got["step"] == ref["step"] == 300
        scale = abs(ref["sums"][1])
        for k in range(8):
            assert abs(got["sums"][k] - ref["sums"][k]) <= 2e-5 * scale, k
        assert got["max_abs_theta"] <= np.pi * (1 + 1e-6) and ref["max_abs_theta"] <= np.pi * (1 + 1e-6)
