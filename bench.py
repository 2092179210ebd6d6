#!/usr/bin/env python3
"""Throughput benchmark of the lattice Abelian-Higgs hot path on GB300.

One bench step = one pass of the whole hot path over the workload: `diag_every`
leapfrog steps (Eqs. up_pi, up_E, up_phi, up_A of arXiv:1809.00995) followed by
one diagnostics pass (xi_L, xi_W, <v^2>_V, <v^2>_L, <v^2>_omega, Gauss residual).
The default workload is a 1024^3 FP32 lattice in the matter era with s = 1,
diagnostics every 50 steps (FP64 reductions); the metric is site-updates/s.
FP32 workloads with an even diagnostics interval run two leapfrog steps per
kernel pass (AH_FLAG_TWO_STEP, temporal blocking); `--single-step` runs one.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--single-step]
                  [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank evolves its own lattice
(independent seeds): replicas, no collective on the data path; the barrier and
the max-over-ranks timing follow the contract.  `--impl reference` times the
FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (N, precision, era, s, seed, diag_every, description)
    "lattice1024_fp32_matter_s1": (1024, 0, 2, 1.0, 3, 50,
                                   "1024^3 FP32 state, matter era a~tau^2, s=1, lambda0=2, e0=1, dx=0.5, "
                                   "dt=0.1, random-phase init (Philox seed 3), diagnostics every 50 steps"),
    "lattice256_fp32_rad_s0": (256, 0, 1, 0.0, 2, 20,
                               "256^3 FP32 state, radiation era a~tau, s=0, seed 2, diagnostics every 20 steps"),
    "lattice256_fp64_rad_s0": (256, 1, 1, 0.0, 2, 20,
                               "256^3 FP64 state, radiation era a~tau, s=0, seed 2, diagnostics every 20 steps"),
    # the paper's own production case (Sec. 3-4: 512^3, radiation, s=0, diagnostics
    # every 5 steps), for comparison with its Quadro P5000 figures
    "lattice512_fp32_rad_s0_diag5": (512, 0, 1, 0.0, 1, 5,
                                     "512^3 FP32 state, radiation era a~tau, s=0, seed 1, diagnostics every 5 steps"),
    # profiling-sized case of the default workload (3.2 GB state, larger than L2)
    "lattice384_fp32_matter_s1": (384, 0, 2, 1.0, 3, 50,
                                  "384^3 FP32 state, matter era a~tau^2, s=1, seed 3, diagnostics every 50 steps"),
}
DEFAULT = "lattice1024_fp32_matter_s1"
BYTES_PER_SITE = {0: 80, 1: 160}      # one read + one write of the 10-real state
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--single-step", action="store_true",
                    help="one leapfrog step per kernel pass (default for FP32 workloads with an even "
                         "diagnostics interval: AH_FLAG_TWO_STEP, two steps per pass)")
    ap.add_argument("--variant", default=None,
                    help="step-kernel shape by name (default: autotuned), e.g. ty8_b4_w, or two_ty8_b3 "
                         "in two-step mode")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests of the serving run (the full workload is 500, arriving at 2 per second)")
    ap.add_argument("--no-batch1024", action="store_true",
                    help="skip the batched step on one 1024^3 lattice")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(dist, x, device):
    """The largest of every rank's x (a replica job takes as long as its slowest
    rank); x itself when there is no process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, n_sites, leapfrog_steps, seconds):
    """Whole-job site-updates per second over all replicas."""
    return world * n_sites * leapfrog_steps / seconds


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


# sources of the single-step and the two-step kernel: a traffic record is void
# once any of its kernel's sources changes
KERNEL_SOURCES = {"k_fused": ("k_fused.cu", "fused_common.cuh", "sincos32.cuh"),
                  "k_fused2": ("k_fused2.cu", "k_fused2_tile.cuh", "fused_common.cuh", "sincos32.cuh")}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1809_00995_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def use_two_step(precision, diag_every, single_step=False):
    """Two leapfrog steps per kernel pass (temporal blocking) where the library
    offers it (FP32) and the diagnostics interval is a whole number of passes."""
    return precision == 0 and diag_every % 2 == 0 and not single_step


def traffic_record(kernel, variant):
    """The committed ncu DRAM record of `kernel` if it was taken on the current
    kernel sources and on the shape that ran, else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)[kernel]
        if d.get("sources_sha256_16") != kernel_source_hash(kernel) or d.get("variant") != variant:
            return None
        return d
    except Exception:
        return None


def traffic_per_launch(N, kernel, variant):
    """DRAM bytes per launch of `kernel` on an N^3 lattice: the bytes per site of
    the committed one-launch ncu capture (taken on a lattice of a few GB, see its
    "N") times N^3.  The per-site traffic of this kernel grows little with the
    lattice (halo re-reads that L2 no longer serves), so the scaled figure is a
    slight underestimate on larger lattices."""
    d = traffic_record(kernel, variant)
    return None if d is None else d["dram_bytes_per_site"] * N ** 3


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def cpu_oracle_rate(wl, budget_s=12.0, M=48):
    """Site-updates/s of the FP64 CPU oracle on a bounded sample of the workload: an
    M^3 window of the same lattice (same init, same couplings), stepped until about
    budget_s seconds have passed, plus one diagnostics pass weighted by 1/diag_every."""
    import oracle as O
    N, prec, era, s, seed, diag_every, _ = WORKLOADS[wl]
    p = O.Params(N=N, era=era, s=s, seed=seed)
    f = O.init(p, M=M, origin=(N // 3, N // 5, N // 7))
    O.evolve(p, f, 0, 1)                       # warm (threads, pages)
    n, t0 = 0, time.perf_counter()
    while True:
        O.evolve(p, f, 1 + n % 200, 1)         # stays within the first 200 steps of the run
        n += 1
        if time.perf_counter() - t0 > budget_s * 0.8:
            break
    t_step = (time.perf_counter() - t0) / n
    t1 = time.perf_counter()
    O.observables(p, f, 1 + n)
    t_diag = time.perf_counter() - t1
    rate = M ** 3 / (t_step + t_diag / diag_every)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return rate, cores, "%d^3 window of the %d^3 workload, %d oracle steps (%.2f ms/step) + 1 diagnostics pass " \
                        "(%.1f ms) weighted 1/%d" % (M, N, n, 1e3 * t_step, 1e3 * t_diag, diag_every)


def cpu_oracle_rate_single_thread(wl, budget_s=8.0, M=32):
    """The same measurement on one host core (a child process with OMP_NUM_THREADS=1,
    so that the oracle's OpenMP runtime starts with one thread)."""
    code = ("import json, bench; r, c, smp = bench.cpu_oracle_rate(%r, %r, %d); "
            "print(json.dumps({'value': r, 'cores': c, 'sample': smp}))" % (wl, budget_s, M))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=300)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as e:                      # reported, not fatal: the main line still prints
        return {"unavailable": str(e)[:200]}


def batch_configs(ah, count=64, seed=4):
    """The batched-ensemble workload: N ~ U{64, 96, 128, 192, 256}, era ~ U{radiation,
    matter}, s ~ U{0, 1} from a fixed-seed host RNG, seeds 100..163, each run to
    tau = N dx / 2 (FP32)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    cfgs = []
    for i in range(count):
        N = int(rng.choice([64, 96, 128, 192, 256]))
        era = int(rng.choice([ah.AH_RADIATION, ah.AH_MATTER]))
        s = float(rng.choice([0.0, 1.0]))
        cfgs.append(ah.config(N, era=era, s=s, seed=100 + i, precision=ah.AH_FP32))
    return cfgs


def run_batch(ah, torch):
    cfgs = batch_configs(ah)
    # AH_BATCH_TWO_STEP pairs the steps of lattices of side >= 512 only: every
    # lattice of this ensemble (N <= 256) takes one step per launch
    series, st = ah.ah_batch_run(cfgs, flags=ah.AH_BATCH_AUTOTUNE | ah.AH_BATCH_TWO_STEP, series_cap=2)
    rate = st["site_updates"] / st["seconds"]
    # looping the single-lattice paths over a sample of the same lattices
    sample = sorted(range(len(cfgs)), key=lambda i: cfgs[i].N)[::8][:6]

    def loop(kernel):
        su, t = 0.0, 0.0
        for i in sample:
            c = cfgs[i]
            n = int(round((c.tau_end - c.tau0) / c.dt))
            g = ah.Sim(c.N, era=c.era, s=c.s, seed=c.seed, kernel=kernel)
            g.sync()
            t0 = time.perf_counter()
            g.step(n)
            g.observables()
            t += time.perf_counter() - t0
            su += c.N ** 3 * n
            g.close()
        return su / t

    loop_fused = loop(ah.AH_KERNEL_FUSED)
    loop_plain = loop(ah.AH_KERNEL_PLAIN)
    return {"workload": "64 FP32 lattices, N ~ U{64,96,128,192,256}, era and s uniform, seeds 100-163, "
                        "each to tau = N dx / 2; diagnostics at start and end",
            "mode": "AH_BATCH_TWO_STEP | AH_BATCH_AUTOTUNE (every lattice here, N <= 256, one step per launch)",
            "sims_per_hour": st["sims_per_hour"], "site_updates_per_s": rate, "seconds": st["seconds"],
            "setup_seconds": st["setup_seconds"], "site_updates": st["site_updates"], "shape": st["shape"],
            "launches": st["launches"], "graph_replays": st["rounds"],
            "loop_fused_site_updates_per_s": loop_fused, "loop_plain_fp32_site_updates_per_s": loop_plain,
            "speedup_vs_loop_plain": rate / loop_plain, "speedup_vs_loop_fused": rate / loop_fused,
            "loop_sample": "%d of the lattices (N = %s), each alone to its end" % (
                len(sample), ",".join(str(cfgs[i].N) for i in sample))}


def run_batch1024(ah, peak, flags=0, N=1024, short=40, long=100):
    """The batched engine's step on one N^3 FP32 lattice (matter era, s = 1, seed 3):
    two ah_batch_run jobs of `short` and `long` steps; their difference in wall
    time over the difference in steps is the time of one batched step (setup and
    the diagnostics at start and end cancel)."""
    def job(n):
        c = ah.config(N, era=ah.AH_MATTER, s=1.0, seed=3, precision=ah.AH_FP32)
        c.tau_end = c.tau0 + n * c.dt
        c.tau_ref = N * c.dx / 2.0
        _, st = ah.ah_batch_run([c], flags=flags, series_cap=2)
        return st
    job(4)                                    # warm-up: kernels configured, pool grown
    a, b = job(short), job(long)
    ms = (b["seconds"] - a["seconds"]) / (long - short) * 1e3
    gbs = 80.0 * N ** 3 / (ms / 1e3) / 1e9
    return {"workload": "one %d^3 FP32 lattice through ah_batch_run (matter era, s = 1, seed 3)" % N,
            "mode": "two leapfrog steps per launch" if flags & ah.AH_BATCH_TWO_STEP else "one step per launch",
            "ms_per_step": ms, "site_updates_per_s": N ** 3 / (ms / 1e3), "alg_gbs": gbs, "peak_gbs": peak,
            "hbm_frac": gbs / peak, "effective": bool(flags & ah.AH_BATCH_TWO_STEP),
            "launches_per_step": (b["launches"] - a["launches"]) / (long - short),
            "weak_field_launches": b.get("weak_field_launches", 0),
            "method": "difference of %d- and %d-step batch jobs (wall clock), 80 B per site-update" % (long, short)}


def run_serve(ah, nreq, rate=2.0, seed=5, budget=150 << 30):
    """Poisson arrivals (mean `rate`/s) of runs with N in {64,128,192,256,384}
    (weights .3/.3/.2/.15/.05), era and s uniform, fresh seeds, each to
    tau = N dx / 2, diagnostics every 20 steps, 150 GB budget."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.choice([64, 128, 192, 256, 384], size=nreq, p=[0.3, 0.3, 0.2, 0.15, 0.05])
    gaps = rng.exponential(1.0 / rate, size=nreq)
    cfgs = [ah.config(int(N), era=int(rng.choice([ah.AH_RADIATION, ah.AH_MATTER])),
                      s=float(rng.choice([0.0, 1.0])), seed=1000 + i, diag_every=20, precision=ah.AH_FP32)
            for i, N in enumerate(Ns)]
    ids = []
    with ah.Server(budget, max_slots=64, flags=ah.AH_BATCH_TWO_STEP) as srv:
        t0 = time.perf_counter()
        t_next = 0.0
        for c, gap in zip(cfgs, gaps):
            t_next += gap
            d = t_next - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            ids.append(srv.submit(c))
        res = []
        for rid in ids:
            while True:
                r = srv.poll(rid)
                if r is not None:
                    res.append(r)
                    break
                time.sleep(0.002)
        st = srv.stats()
    lat = np.array([td - ts for _, ts, td in res])
    first = min(ts for _, ts, _ in res)
    last = max(td for _, _, td in res)
    su = sum(c.N ** 3 * int(round((c.tau_end - c.tau0) / c.dt)) for c in cfgs)
    return {"workload": "Poisson arrivals, mean 2/s, N in {64,128,192,256,384} (weights .3/.3/.2/.15/.05), "
                        "era and s uniform, each to tau = N dx / 2, diagnostics every 20 steps, 150 GB budget",
            "mode": "AH_BATCH_TWO_STEP (pairs for N >= 512: none in this workload, one step per launch)",
            "requests": nreq, "sims_per_hour": nreq * 3600.0 / (last - first),
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "site_updates_per_s": su / (last - first),
            "offered_site_updates_per_s": su / float(np.sum(gaps)), "launches": st["launches"],
            "sample": "%d requests (the full workload is 500)" % nreq if nreq < 500 else "full 500 requests"}


def reference_arm(a, wl, rank, world):
    """The CPU oracle as it stands, timed on the host cores; rank 0 only."""
    if rank != 0:
        return
    import oracle as O
    N, prec, era, s, seed, diag_every, desc = WORKLOADS[wl]
    M = 40
    p = O.Params(N=N, era=era, s=s, seed=seed)
    f = O.init(p, M=M, origin=(N // 3, N // 5, N // 7))
    n = 0

    def one():
        nonlocal n
        O.evolve(p, f, n, diag_every)
        n += diag_every
        O.observables(p, f, n)

    for _ in range(a.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        one()
    t = time.perf_counter() - t0
    value = M ** 3 * diag_every * a.steps / t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = "%d^3 window of the workload per step: %d oracle leapfrog steps + 1 diagnostics pass" % (M, diag_every)
    print(json.dumps({
        "impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl, "description": desc, "N": N, "diag_every": diag_every},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value, "unit": "site-updates/s"},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    a = parse()
    rank, local_rank, world = dist_env()
    wl = a.workload
    if a.impl == "reference":
        return reference_arm(a, wl, rank, world)

    import torch
    import paper_1809_00995_gb300 as ah
    from paper_1809_00995_gb300 import _build

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()

    def barrier():
        if dist:
            dist.barrier()

    N, prec, era, s, seed, diag_every, desc = WORKLOADS[wl]
    n_sites = N ** 3
    stream = torch.cuda.Stream()
    two_step = use_two_step(prec, diag_every, a.single_step)
    mode = ah.AH_FLAG_TWO_STEP if two_step else 0
    g = ah.Sim(N, precision=prec, kernel=ah.AH_KERNEL_FUSED, era=era, s=s, seed=seed + 1000 * rank,
               flags=mode | (0 if a.variant else ah.AH_FLAG_AUTOTUNE))
    if a.variant:
        names = {}
        for v in range(g.info["n_variants"]):
            try:
                g.set_variant(v)
                names[g.info["variant_name"]] = v
            except ah.AhError:
                pass
        g.set_variant(names[a.variant])
    ah.ah_set_stream(g.h, stream.cuda_stream)
    info = g.info

    def bench_step(ev_a=None, ev_b=None):
        if ev_a is not None:
            ev_a.record(stream)
        g.step(diag_every)
        if ev_b is not None:
            ev_b.record(stream)
        return g.observables()

    for _ in range(a.warmup):
        obs = bench_step()
    torch.cuda.synchronize()

    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    weak0 = g.info["weak_field_launches"]
    start.record(stream)
    for k in range(a.steps):
        obs = bench_step(*ev[k])
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    t_ms = start.elapsed_time(end)
    step_ms = sum(x.elapsed_time(y) for x, y in ev)
    t_max = max_over_ranks(dist, t_ms, "cuda")
    value = job_value(world, n_sites, diag_every * a.steps, t_max / 1e3)

    variant_name = info["variant_name"]
    weak_launches = g.info["weak_field_launches"] - weak0
    g.close()

    # end to end through the public C ABI, host clock: one whole job as a user
    # runs it -- ah_create_ex from a host ah_config (device allocation, Philox
    # initial state), then per bench step ah_step(diag_every) and
    # ah_observables into a host ah_obs (device-to-host copy, stream sync),
    # then ah_destroy.  The state stays resident between steps, so no step has
    # host-to-device input bytes; the job's only input is the config.
    import ctypes
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    cfg_e2e = ah.config(N, precision=prec, kernel=ah.AH_KERNEL_FUSED, era=era, s=s, seed=seed + 1000 * rank,
                        flags=mode | (0 if a.variant else ah.AH_FLAG_AUTOTUNE))
    h = ah.ah_create_ex(cfg_e2e)
    try:
        if a.variant:
            ah.ah_set_variant(h, names[a.variant])
        for _ in range(a.steps):
            ah.ah_step(h, diag_every)
            obs_e2e = ah.ah_observables(h)
    finally:
        ah.ah_destroy(h)
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    e2e_value = job_value(world, n_sites, diag_every * a.steps, t_e2e)
    d2h = ctypes.sizeof(ah.ah_obs)
    final_obs = obs_e2e

    # one launch = one leapfrog step, or two in two-step mode.  Algorithmic
    # bytes: 80 B (FP32) / 160 B (FP64) per site-update whatever the kernel, so
    # a two-step launch counts 2 x that; it moves the state once, so its
    # `achieved` is an effective bandwidth and its DRAM traffic is about half.
    steps_per_launch = 2 if two_step else 1
    avg_launch_s = step_ms / 1e3 / (a.steps * diag_every) * steps_per_launch
    alg_bytes = BYTES_PER_SITE[prec] * n_sites * steps_per_launch
    peak, peak_src = peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    kname = "k_fused2" if two_step else "k_fused"
    tr = traffic_per_launch(N, kname, variant_name)
    trec = traffic_record(kname, variant_name)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": tr,
                "traffic_source": None if trec is None else
                "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at %d^3 (%.2f B/site), "
                "scaled to %d^3 by the site count" % (trec["N"], trec["dram_bytes_per_site"], N),
                "kernel": ("fused step, shape %s (one leapfrog step per launch)" % variant_name if not two_step else
                           "two-step fused kernel, shape %s (two leapfrog steps per launch; %d of the %d timed "
                           "launches the form for weak gauge fields)"
                           % (variant_name, weak_launches, a.steps * diag_every // steps_per_launch)),
                "peak_source": peak_src,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_launch_s * 1e3,
                "step_share_of_time": step_ms / t_ms}
    if two_step:
        roofline["effective"] = True
        roofline["dram_state_bytes_per_launch"] = BYTES_PER_SITE[prec] * n_sites
        roofline["dram_frac"] = BYTES_PER_SITE[prec] * n_sites / avg_launch_s / 1e9 / peak

    plain = None
    if rank == 0 and not a.no_plain:
        # the plain FP64 single-lattice path (the paper's three-kernel structure) on
        # the same lattice size: the speed-up denominator
        try:
            h = ah.Sim(N, precision=ah.AH_FP64, kernel=ah.AH_KERNEL_PLAIN, era=era, s=s, seed=seed)
            ah.ah_set_stream(h.h, stream.cuda_stream)
            h.step(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            np_ = 3
            e0.record(stream)
            h.step(np_)
            e1.record(stream)
            torch.cuda.synchronize()
            tp = e0.elapsed_time(e1) / 1e3
            h.close()
            pv = n_sites * np_ / tp
            plain = {"value": pv, "unit": "site-updates/s", "steps": np_, "dtype": "f64",
                     "kernel": "plain (Pi kick, E kick, drift)", "speedup_of_value_over_plain": value / pv}
        except ah.AhError as e:
            plain = {"unavailable": str(e)}

    batch = serve = batch1024 = None
    if rank == 0 and not a.no_batch:
        batch = run_batch(ah, torch)
    if rank == 0 and not a.no_batch1024:
        batch1024 = run_batch1024(ah, peak, flags=ah.AH_BATCH_TWO_STEP)
        batch1024["one_step_per_launch"] = run_batch1024(ah, peak, flags=0)
    if rank == 0 and not a.no_serve:
        serve = run_serve(ah, a.serve_requests)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        rate, cores, sample = cpu_oracle_rate(wl)
        cpu = {"value": rate, "unit": "site-updates/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": cpu_oracle_rate_single_thread(wl)}

    if rank == 0:
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == 0 else "f64", "data": "synthetic",
            "config": {"workload": wl, "description": desc, "N": N, "diag_every": diag_every,
                       "leapfrog_steps_per_bench_step": diag_every,
                       "leapfrog_steps_per_launch": steps_per_launch,
                       "l2": "inputs larger than L2 (%.1f GB state)" % (info["state_bytes"] / 1e9),
                       "parallelism": "replicas" if world > 1 else "single"},
            "hbm_gbs_effective": achieved,
            "roofline": roofline,
            # the rest of a bench step: one whole-lattice diagnostics pass (k_fused_diag
            # tile walk, ordered sum, near-cut fix-up) and its read-back to the host
            "diag_pass": {"ms_per_pass": (t_ms - step_ms) / a.steps, "share_of_time": 1.0 - step_ms / t_ms,
                          "bound": "issue (FP32 arithmetic of the estimators, windings and double-float "
                                   "Gauss residual; one read of the state)"},
            "cpu_baseline": cpu,
            "plain_fp64": plain,
            "e2e": {"value": e2e_value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": d2h, "h2d_bytes_per_job": ctypes.sizeof(ah.ah_config),
                    "timed": "ah_create_ex + %d x (ah_step(%d) + ah_observables to host) + ah_destroy, host clock"
                             % (a.steps, diag_every)},
            # per bench step: the step launches and the diagnostics pass (tile
            # walk, ordered sum, near-cut fix-up)
            "gpu_launches": a.steps * (diag_every * info["step_launches"] // steps_per_launch + 3),
            "batch": batch,
            "batch1024": batch1024,
            "serve": serve,
            "clocks": clocks,
            "final_obs": {k: final_obs[k] for k in ("step", "tau", "xi_L", "xi_W", "v2_V", "v2_L", "v2_omega",
                                                     "gauss_rel", "max_abs_theta")},
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
