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


# ------------------------------------------------------------- fields vs the oracle
TOL32 = 1e-5     # per component max|f_gpu - f_ref| / max(max|f_ref|, 1), FP32 state, 20 steps


def rel_err(got, ref):
    return [float(np.max(np.abs(got[c] - ref[c])) / max(np.max(np.abs(ref[c])), 1.0)) for c in range(10)]


def short_config(N, era, s, seed, nsteps, **kw):
    """A run of `nsteps` steps from tau0 = 1 with the scale-factor normalisation of
    the full run (tau_ref = N dx / 2)."""
    c = ah.config(N, era=era, s=s, seed=seed, **kw)
    c.tau_ref = N * c.dx / 2.0
    c.tau_end = c.tau0 + nsteps * c.dt
    return c


def oracle_fields(cfg, nsteps, M=None, origin=(0, 0, 0)):
    """The oracle's evolution of the FP32 state's initial values (a window of M^3
    sites at `origin`, default the whole lattice) over nsteps steps."""
    p = O.Params(N=cfg.N, era=cfg.era, s=cfg.s, seed=cfg.seed, tau_ref=cfg.tau_ref,
                 wrap_theta=bool(cfg.flags & ah.AH_FLAG_WRAP_THETA),
                 core_growth=bool(cfg.flags & ah.AH_FLAG_CORE_GROWTH))
    f = O.init(p, M=M, origin=origin).astype(np.float32).astype(np.float64)
    return O.evolve(p, f, 0, nsteps), p


@pytest.mark.parametrize("paired,flags", [("none", 0), ("all", 0), ("some", ah.AH_BATCH_AUTOTUNE)])
def test_batch_fields_match_oracle(paired, flags):
    """Every lattice of a mixed batch (ragged sides that leave partial tiles and z
    chunks, both eras, s = 0 and 1, 20 or 21 steps so that a lattice stepped in
    pairs also ends with one single step) equals the oracle field by field after
    its run: per component within 1e-5 of max(max|f|, 1) (FP32 state, Eqs.
    up_pi, up_E, up_phi, up_A), and its final observables equal the oracle's on
    the returned snapshot (sums to the FP32 tolerance, windings exactly).  The
    lattices are stepped one step per launch, all in pairs (two-step passes,
    AH_FLAG_TWO_STEP), or half of them in pairs."""
    Ns = [12, 17, 20, 33, 24, 9]
    cfgs = []
    for i, N in enumerate(Ns):
        era, s = ERAS[i % len(ERAS)]
        pair = paired == "all" or (paired == "some" and i % 3 != 1)
        cfgs.append(short_config(N, era, s, 300 + i, 20 + (i % 2), diag_every=0,
                                 flags=ah.AH_FLAG_TWO_STEP if pair else 0))
    wins = [(i, 0, 0, 0, c.N, c.N, c.N) for i, c in enumerate(cfgs)]
    series, st, fields = ah.ah_batch_run_ex(cfgs, wins, flags=flags)
    assert st["launches"] > 0
    for i, c in enumerate(cfgs):
        n = 20 + (i % 2)
        ref, p = oracle_fields(c, n)
        err = rel_err(fields[i], ref)
        assert max(err) <= TOL32, (c.N, err)
        go = series[i][-1]
        assert go["step"] == n
        oo = O.observables(p, fields[i], n)
        S1 = abs(oo["sum_rho"])
        for k, name in enumerate(["sum_L", "sum_rho", "sum_p", "sum_K", "sum_G2", "sum_V", "sum_Eel", "sum_B"]):
            assert abs(go["sums"][k] - oo[name]) <= 1e-5 * abs(oo[name]) + 2e-6 * S1, (c.N, name)
        assert list(go["wind_abs_plane"]) == list(oo["sum_abs_W_plane"])
        assert go["n_pierced"] == oo["n_pierced"]


def test_batch_two_step_equals_one_step_per_launch():
    """Two steps per batched launch and one step per launch evaluate the same
    formulas: the same lattices agree to FP32 rounding (contractions may differ),
    including a run with compact link phases and one with core growth."""
    cfgs = [short_config(20, ah.AH_MATTER, 1.0, 41, 30, diag_every=0),
            short_config(27, ah.AH_RADIATION, 0.0, 42, 31, diag_every=0, flags=ah.AH_FLAG_WRAP_THETA),
            short_config(16, ah.AH_RADIATION, 0.0, 43, 25, diag_every=0, flags=ah.AH_FLAG_CORE_GROWTH)]
    cfgs[2].tau_ref = cfgs[2].tau0 + 1.25       # the switch from s to 1 falls inside the run
    wins = [(i, 0, 0, 0, c.N, c.N, c.N) for i, c in enumerate(cfgs)]
    _, _, one = ah.ah_batch_run_ex(cfgs, wins, flags=0)
    for c in cfgs:
        c.flags |= ah.AH_FLAG_TWO_STEP
    _, st, two = ah.ah_batch_run_ex(cfgs, wins, flags=0)
    for a, b in zip(one, two):
        assert max(rel_err(b, a)) <= 1e-5
    # rounds of 25, 6 and 1 steps (each lattice keeps its steps in pairs and
    # takes a single step only one step before its end): 12 + 3 two-step passes
    # and 2 single-step launches, two kernels (step and advance) per launch
    assert st["launches"] == 2 * (12 + 1 + 3 + 1)


def test_batch_1024cubed_light_cone_windows():
    """A 1024^3 FP32 lattice (matter era, s = 1, seed 3: the configuration of the
    throughput target) run through the batched engine with AH_BATCH_TWO_STEP
    (lattices of side >= 512 in pairs, each launched with its own two-step grid)
    and autotuned shapes, beside a small lattice stepped in pairs by the
    persistent two-step pass and one stepped one step per launch: after 20 steps
    three 16^3 windows (two across the periodic seam) equal the oracle's
    evolution of the (16 + 2 * 20)^3 windows of the same initial lattice (the
    big lattice's passes take the kernel for weak gauge fields, as the bench's
    do); the small lattices equal the oracle whole."""
    N, k, b = 1024, 20, 16
    big = short_config(N, ah.AH_MATTER, 1.0, 3, k, diag_every=0)
    # the 24^3 lattice is paired too (batched two-step pass); the 13^3 one takes
    # one step per launch and ends on an odd step
    small = [short_config(24, ah.AH_RADIATION, 0.0, 5, k, diag_every=0, flags=ah.AH_FLAG_TWO_STEP),
             short_config(13, ah.AH_MATTER, 0.0, 6, k + 1, diag_every=0)]
    cfgs = [big] + small
    orgs = [(1016, 5, 1019), (300, 1010, 7), (511, 512, 640)]
    wins = [(0, *o, b, b, b) for o in orgs] + [(1, 0, 0, 0, 24, 24, 24), (2, 0, 0, 0, 13, 13, 13)]
    series, st, fields = ah.ah_batch_run_ex(cfgs, wins, flags=ah.AH_BATCH_TWO_STEP | ah.AH_BATCH_AUTOTUNE,
                                            series_cap=2)
    # the observables at step 0 found max |theta| = 0: all ten passes of the
    # 1024^3 lattice take the kernel for weak gauge fields
    assert st["weak_field_launches"] == k // 2
    for w, org in enumerate(orgs):
        M = b + 2 * k
        ref, _ = oracle_fields(big, k, M=M, origin=[(o - k) % N for o in org])
        assert max(rel_err(fields[w], ref[:, k:k + b, k:k + b, k:k + b])) <= TOL32, org
    for j, c in enumerate(small):
        ref, _ = oracle_fields(c, k + j)
        assert max(rel_err(fields[3 + j], ref)) <= TOL32, c.N
    o = series[0][-1]
    assert o["step"] == k and o["n_sites"] == N ** 3 and o["nonfinite"] == 0 and o["gauss_rel"] < 1e-5


def test_batch_large_paired_lattice_ending_before_the_others():
    """A 512^3 lattice stepped in pairs with its own two-step grid (AH_BATCH_TWO_STEP)
    ends after 10 steps while a small lattice runs on to 30: the rounds after its
    end leave it alone, so its final state (an 8^3 window across the seam, against
    the oracle's evolution of the (8 + 2 * 10)^3 window) and its observables are
    those of step 10."""
    N, k, b = 512, 10, 8
    big = short_config(N, ah.AH_RADIATION, 0.0, 8, k, diag_every=0)
    small = short_config(20, ah.AH_MATTER, 1.0, 9, 3 * k, diag_every=4)
    org = (508, 250, 3)
    series, st, fields = ah.ah_batch_run_ex([big, small], [(0, *org, b, b, b), (1, 0, 0, 0, 20, 20, 20)],
                                            flags=ah.AH_BATCH_TWO_STEP, series_cap=16)
    assert st["weak_field_launches"] == k // 2
    ref, _ = oracle_fields(big, k, M=b + 2 * k, origin=[(o - k) % N for o in org])
    assert max(rel_err(fields[0], ref[:, k:k + b, k:k + b, k:k + b])) <= TOL32
    ref_small, _ = oracle_fields(small, 3 * k)
    assert max(rel_err(fields[1], ref_small)) <= TOL32
    assert series[0][-1]["step"] == k and series[1][-1]["step"] == 3 * k


def test_batch_window_arguments_are_checked():
    c = short_config(8, ah.AH_RADIATION, 0.0, 1, 2)
    for w in [(1, 0, 0, 0, 4, 4, 4), (0, 0, 0, 0, 9, 4, 4), (0, 0, 0, 0, 0, 4, 4)]:
        with pytest.raises(ah.AhError) as e:
            ah.ah_batch_run_ex([c], [w])
        assert e.value.status == ah.AH_ERR_ARG


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


@pytest.mark.parametrize("pairs", [False, True])
def test_server_results_same_alone_and_in_the_mix(pairs):
    """Requests arriving while others run are admitted as slots free up, stepped
    together, and each final result equals the same request served alone (also
    when some requests are stepped in pairs, AH_FLAG_TWO_STEP: each keeps its
    own grouping of steps whatever the mix).  One request, admitted while others
    run, returns its final fields, which equal the oracle's run of the same
    configuration."""
    cfgs = mixed_configs([32, 16, 24, 40, 12, 20, 28, 36], diag_every=0, seed0=500)
    probe = short_config(22, ah.AH_MATTER, 1.0, 77, 21, diag_every=0)
    if pairs:
        for c in cfgs[::2] + [probe]:
            c.flags |= ah.AH_FLAG_TWO_STEP
    flags = 0
    with ah.Server(hbm_budget_bytes=8 << 30, max_slots=3, flags=flags) as srv:
        ids = []
        for i, c in enumerate(cfgs):
            ids.append(srv.submit(c))
            if i % 3 == 2:
                time.sleep(0.02)          # later requests arrive while earlier ones run
            if i == 4:
                pid, (pf,) = srv.submit_ex(probe, [(0, 0, 0, 22, 22, 22)])
        results = [wait_done(srv, rid) for rid in ids]
        pobs, _, _ = wait_done(srv, pid)
        ref, p = oracle_fields(probe, 21)
        assert max(rel_err(pf, ref)) <= TOL32
        assert pobs["step"] == 21
        oo = O.observables(p, pf, 21)
        assert list(pobs["wind_abs_plane"]) == list(oo["sum_abs_W_plane"])
        assert abs(pobs["sums"][1] - oo["sum_rho"]) <= 1e-5 * abs(oo["sum_rho"])
        st = srv.stats()
        assert st["completed"] == len(cfgs) + 1 and st["running"] == 0 and st["queued"] == 0
        assert st["hbm_used"] == 0 and st["site_updates"] > 0
    with ah.Server(hbm_budget_bytes=8 << 30, max_slots=1, flags=flags) as srv:
        for c, (obs, ts, td) in zip(cfgs, results):
            assert td >= ts
            alone, _, _ = wait_done(srv, srv.submit(c))
            same_obs(obs, alone)
            close_obs(obs, single_series(c)[-1])


def test_server_large_paired_request_matches_oracle():
    """A 512^3 request stepped in pairs (AH_BATCH_TWO_STEP server: its own two-step
    grid, launched from the server's copy of its state) served beside small
    requests of other lengths: its final fields (an 8^3 window across the seam,
    against the oracle's (8 + 2 * 12)^3 window) and the small ones' equal the
    oracle's."""
    N, k, b = 512, 12, 8
    big = short_config(N, ah.AH_MATTER, 1.0, 21, k, diag_every=0)
    smalls = [short_config(16, ah.AH_RADIATION, 0.0, 22, 2 * k + 1, diag_every=5),
              short_config(20, ah.AH_MATTER, 0.0, 23, 7, diag_every=0)]
    org = (505, 0, 300)
    with ah.Server(hbm_budget_bytes=24 << 30, max_slots=4, flags=ah.AH_BATCH_TWO_STEP) as srv:
        bid, (bf,) = srv.submit_ex(big, [(*org, b, b, b)])
        sids = [srv.submit_ex(c, [(0, 0, 0, c.N, c.N, c.N)]) for c in smalls]
        bobs, _, _ = wait_done(srv, bid)
        for (rid, (f,)), c in zip(sids, smalls):
            obs, _, _ = wait_done(srv, rid)
            n = int(round((c.tau_end - c.tau0) / c.dt))
            ref, _ = oracle_fields(c, n)
            assert max(rel_err(f, ref)) <= TOL32, c.N
            assert obs["step"] == n
    assert bobs["step"] == k
    ref, _ = oracle_fields(big, k, M=b + 2 * k, origin=[(o - k) % N for o in org])
    assert max(rel_err(bf, ref[:, k:k + b, k:k + b, k:k + b])) <= TOL32


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
