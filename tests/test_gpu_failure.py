"""Failure detection on the GPU without a GPU fault (bounded waits).

The TMA-fed step waits on mbarriers for its tensor-map copies; every wait is
bounded and, when it gives up, the kernel records an error word, stops issuing
copies, waits (again bounded) for the copies it still has in flight and
returns, so the context stays usable.  The test injects the failure from the
host (read when a simulation is created): AH_TMA_DROP_COPY leaves one copy per
CTA unissued, so a barrier that nothing completes is waited on, and
AH_TMA_WAIT_LIMIT_CYCLES shortens the bound to about a millisecond."""
import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah

pytestmark = pytest.mark.gpu


def _variant_index(g, name):
    for v in range(g.info["n_variants"]):
        try:
            g.set_variant(v)
        except ah.AhError:
            continue
        if g.info["variant_name"] == name:
            return v
    raise LookupError(name)


def test_tma_wait_timeout_is_reported_and_the_device_stays_usable(monkeypatch):
    N = 64
    monkeypatch.setenv("AH_TMA_DROP_COPY", "1")
    monkeypatch.setenv("AH_TMA_WAIT_LIMIT_CYCLES", str(1 << 21))
    g = ah.Sim(N, precision=ah.AH_FP32, kernel=ah.AH_KERNEL_FUSED, seed=3)
    monkeypatch.delenv("AH_TMA_DROP_COPY")
    monkeypatch.delenv("AH_TMA_WAIT_LIMIT_CYCLES")
    try:
        g.set_variant(_variant_index(g, "tma_b3"))
        g.step(2)
        with pytest.raises(ah.AhError) as e:
            g.sync()
        assert e.value.status == ah.AH_ERR_TIMEOUT
        g.sync()                          # the error word was read and cleared
    finally:
        g.close()
    # the same kernel with the default bound, on the same device, matches the oracle
    p = O.Params(N=N, era=O.RADIATION, seed=3)
    with ah.Sim(N, precision=ah.AH_FP32, kernel=ah.AH_KERNEL_FUSED, seed=3) as h:
        h.set_variant(_variant_index(h, "tma_b3"))
        f0 = h.fields()
        h.step(20)
        h.sync()
        got = h.fields()
    ref = O.evolve(p, f0, 0, 20)
    err = max(float(np.max(np.abs(got[c] - ref[c])) / max(np.max(np.abs(ref[c])), 1.0)) for c in range(10))
    assert err <= 1e-5
