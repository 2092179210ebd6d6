"""Batched ensembles and the continuous-batching server (GPU).

A lattice run inside a batch, or admitted by the server while others run, must
give exactly the observables of the same configuration run alone through the
same batched path (per-site arithmetic does not depend on the mix), and agree
with the single-lattice path (ah_step, another kernel instantiation whose
floating-point contraction may differ in the last bits) and the oracle within
the FP32 tolerance.
"""
import time

import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah

pytestmark = pytest.mark.gpu

ERAS = [(ah.AH_RADIATION, 0.0), (ah.AH_MATTER, 1.0), (ah.AH_RADIATION, 1.0), (ah.AH_MATTER, 0.0)]


def mixed_configs(Ns, diag_every=5, seed0=100):
    cfgs = []
    for i, N in enumerate(Ns):
        era, s = ERAS[i % len(ERAS)]
        cfgs.append(ah.config(N, era=era, s=s, seed=seed0 + i, diag_every=diag_every))
    return cfgs


def single_series(cfg):
    """The same run alone through ah_step / ah_observables (fused shape 0)."""
    out = []
    with ah.Sim(cfg.N, era=cfg.era, s=cfg.s, seed=cfg.seed, kernel=ah.AH_KERNEL_FUSED) as g:
        g.set_variant(0)
        nsteps = int(round((cfg.tau_end - cfg.tau0) / cfg.dt))
        out.append(g.observables())
        n = 0
        while n < nsteps:
            nxt = min(nsteps, (n // cfg.diag_every + 1) * cfg.diag_every) if cfg.diag_every else nsteps
            g.step(nxt - n)
            n = nxt
            out.append(g.observables())
    return out


def same_obs(a, b):
    assert a["step"] == b["step"]
    assert a["sums"] == b["sums"], (a["step"], a["sums"], b["sums"])
    assert a["wind_abs_plane"] == b["wind_abs_plane"] and a["n_pierced"] == b["n_pierced"]


def close_obs(a, b, rtol=2e-5):
    assert a["step"] == b["step"]
    scale = abs(b["sums"][1])
    for k in range(8):
        assert abs(a["sums"][k] - b["sums"][k]) <= rtol * scale, (a["step"], k)


@pytest.mark.parametrize("flags", [0, ah.AH_BATCH_NO_GRAPH, ah.AH_BATCH_AUTOTUNE])
def test_batch_same_alone_and_in_the_mix(flags):
    Ns = [16, 24, 12, 32, 20, 40, 18]
    cfgs = mixed_configs(Ns)
    series, stats = ah.ah_batch_run(cfgs, flags=flags & ~ah.AH_BATCH_AUTOTUNE)
    assert stats["site_updates"] > 0 and stats["seconds"] > 0 and stats["launches"] > 0
    for cfg, ser in zip(cfgs, series):
        alone, _ = ah.ah_batch_run([cfg], flags=flags & ~ah.AH_BATCH_AUTOTUNE)
        assert len(ser) == len(alone[0])
        for a, b in zip(ser, alone[0]):
            same_obs(a, b)
        assert ser[-1]["tau"] == pytest.approx(cfg.tau_end)
    if flags & ah.AH_BATCH_AUTOTUNE:       # any tuned shape: the same physics to FP32 tolerance
        tuned, st = ah.ah_batch_run(cfgs, flags=flags)
        for a_ser, b_ser in zip(tuned, series):
            for a, b in zip(a_ser, b_ser):
                close_obs(a, b)


def test_batch_close_to_single_path():
    cfgs = mixed_configs([16, 24, 12, 20])
    series, _ = ah.ah_batch_run(cfgs)
    for cfg, ser in zip(cfgs, series):
        ref = single_series(cfg)
        assert len(ser) == len(ref)
        for a, b in zip(ser, ref):
            close_obs(a, b)
            assert a["wind_abs_plane"] == b["wind_abs_plane"] or a["step"] > 0


def test_batch_matches_oracle_for_one_lattice():
    """End-to-end: a lattice run inside a batch equals the oracle's run of the same
    configuration, within the FP32 diagnostic tolerance, at its last diagnostic."""
    cfgs = mixed_configs([16, 24, 12], diag_every=0)
    series, _ = ah.ah_batch_run(cfgs)
    cfg = cfgs[0]
    p = O.Params(N=cfg.N, era=cfg.era, s=cfg.s, seed=cfg.seed)
    f = O.init(p).astype(np.float32).astype(np.float64)
    nsteps = int(round((cfg.tau_end - cfg.tau0) / cfg.dt))
    O.evolve(p, f, 0, nsteps)
    oo = O.observables(p, f, nsteps)
    go = series[0][-1]
    rho = oo["sum_rho"]
    for k, name in enumerate(["sum_L", "sum_rho", "sum_p", "sum_K", "sum_G2", "sum_V", "sum_Eel", "sum_B"]):
        assert abs(go["sums"][k] - oo[name]) <= 1e-4 * abs(rho), name


@pytest.mark.parametrize("N", [458, 512])
def test_batch_diagnostics_of_sides_with_large_diag_grids(N):
    """The whole-lattice diagnostics pass takes its z-chunk count from N, so many
    sides need more CTAs (one partial each) than the largest accepted side (512^3:
    8192, 1290^3: 6642).  A batch of such a lattice gives the single-lattice
    observables of the same state: at step 0 exactly, after 4 steps to the FP32
    tolerance."""
    cfg = ah.config(N, era=ah.AH_RADIATION, s=0.0, seed=9, diag_every=0)
    cfg.tau_end = cfg.tau0 + 4 * cfg.dt
    series, _ = ah.ah_batch_run([cfg])
    ref = single_series(cfg)
    assert len(series[0]) == len(ref) == 2
    same_obs(series[0][0], ref[0])
    close_obs(series[0][-1], ref[-1])


def test_batch_rejects_bad_configs():
    with pytest.raises(ah.AhError) as e:
        ah.ah_batch_run([ah.config(16, precision=ah.AH_FP64)])
    assert e.value.status == ah.AH_ERR_ARG
    with pytest.raises(ah.AhError) as e:
        ah.ah_batch_run([ah.config(16, diag_every=-1)])
    assert e.value.status == ah.AH_ERR_ARG


def wait_done(srv, rid, timeout=120.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = srv.poll(rid)
        if r is not None:
            return r
        time.sleep(0.005)
    raise TimeoutError(rid)


def test_server_results_same_alone_and_in_the_mix():
    """Requests arriving while others run are admitted as slots free up, stepped
    together, and each final result equals the same request served alone."""
    cfgs = mixed_configs([32, 16, 24, 40, 12, 20, 28, 36], diag_every=0, seed0=500)
    with ah.Server(hbm_budget_bytes=8 << 30, max_slots=3) as srv:
        ids = []
        for i, c in enumerate(cfgs):
            ids.append(srv.submit(c))
            if i % 3 == 2:
                time.sleep(0.02)          # later requests arrive while earlier ones run
        results = [wait_done(srv, rid) for rid in ids]
        st = srv.stats()
        assert st["completed"] == len(cfgs) and st["running"] == 0 and st["queued"] == 0
        assert st["hbm_used"] == 0 and st["site_updates"] > 0
    with ah.Server(hbm_budget_bytes=8 << 30, max_slots=1) as srv:
        for c, (obs, ts, td) in zip(cfgs, results):
            assert td >= ts
            alone, _, _ = wait_done(srv, srv.submit(c))
            same_obs(obs, alone)
            close_obs(obs, single_series(c)[-1])


def test_server_budget_and_cancel():
    with ah.Server(hbm_budget_bytes=64 << 20, max_slots=4) as srv:
        with pytest.raises(ah.AhError) as e:
            srv.submit(ah.config(128))          # 128^3 FP32 state > 64 MB: can never fit
        assert e.value.status == ah.AH_ERR_OOM
        a = srv.submit(ah.config(48, seed=1))
        b = srv.submit(ah.config(48, seed=2))
        srv.cancel(b)
        with pytest.raises(ah.AhError) as e:
            srv.poll(b)
        assert e.value.status == ah.AH_ERR_CANCELLED
        obs, _, _ = wait_done(srv, a)
        assert obs["step"] == int(round((ah.config(48).tau_end - 1.0) / 0.1))
        with pytest.raises(ah.AhError) as e:
            srv.poll(123456)
        assert e.value.status == ah.AH_ERR_NOTFOUND


def test_server_device_failure_fails_every_request(monkeypatch):
    """Failure detection without a GPU fault: the server's step call reports a
    (host-side fake) device error after two rounds; every running and queued
    request then fails with AH_ERR_CUDA instead of staying busy, later
    submissions are refused with AH_ERR_CUDA, and the server shuts down cleanly."""
    monkeypatch.setenv("AH_FAKE_DEVICE_FAILURE_AFTER_ROUNDS", "2")
    srv = ah.Server(hbm_budget_bytes=8 << 30, max_slots=2)
    monkeypatch.delenv("AH_FAKE_DEVICE_FAILURE_AFTER_ROUNDS")
    try:
        ids = [srv.submit(ah.config(48, seed=70 + i)) for i in range(5)]    # 310 steps each: many rounds
        for rid in ids:
            t0 = time.time()
            while True:
                try:
                    r = srv.poll(rid)
                except ah.AhError as e:
                    assert e.status == ah.AH_ERR_CUDA
                    break
                assert r is None, "a request completed although the device failed"
                assert time.time() - t0 < 60
                time.sleep(0.005)
        st = srv.stats()
        assert st["running"] == 0 and st["queued"] == 0 and st["hbm_used"] == 0
        with pytest.raises(ah.AhError) as e:
            srv.submit(ah.config(16))
        assert e.value.status == ah.AH_ERR_CUDA
    finally:
        srv.close()
    # a fresh server on the same device works
    with ah.Server(hbm_budget_bytes=8 << 30, max_slots=2) as ok:
        obs, _, _ = wait_done(ok, ok.submit(ah.config(16, seed=1)))
        assert obs["nonfinite"] == 0
