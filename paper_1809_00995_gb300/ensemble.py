"""Scaling ensembles of string networks (Sec. 4 of arXiv:1809.00995, Table 3).

A case (era, s, schedule) is run for several seeds as one batched job through
ah_batch_run; each run's diagnostic series gives

  xi_dot_L, xi_dot_W  least-squares slopes d xi / d tau of the Lagrangian and
                      winding mean string separations (Eqs. defXiV2, 9) over
                      the scaling window,
  v2_V, v2_L, v2_w    the mean over the same window of the three velocity
                      estimators (Eqs. defR, defEoS),

and the case reports the mean and the standard deviation over seeds.  The
paper does not state its window; this module takes the second half of the
run, tau in [tau0 + f (tau_end - tau0), tau_end] with f = 1/2 by default.

Command line (one GPU):
    python -m paper_1809_00995_gb300.ensemble --N 512 --seeds 5
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

# name: (era, s, switch): with a switch fraction f the run uses the schedule of
# AH_FLAG_CORE_GROWTH with tau_ref = f tau_end, i.e. fixed comoving width
# (s = 0) up to tau_ref and the true equations (s = 1) after it, so the whole
# scaling window (second half) evolves with s = 1 while the core shrinks to
# half its width by tau_end.  (A growing core, s = -1 from tau0 = 1, needs
# a(tau0)^-2 ~ (tau_ref / tau0)^2 in the stiff mass and is refused by the
# stability check for any tau_ref that keeps the cores resolved at tau_end.)
CASES = {
    "radiation_s0": (1, 0.0, None),
    "matter_s0": (2, 0.0, None),
    "radiation_s1": (1, 0.0, 0.5),
}


def fit_slope(t, y):
    """Least-squares slope and coefficient of determination of y(t)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    tm, ym = t.mean(), y.mean()
    stt = np.sum((t - tm) ** 2)
    slope = float(np.sum((t - tm) * (y - ym)) / stt)
    resid = y - (ym + slope * (t - tm))
    syy = np.sum((y - ym) ** 2)
    r2 = float(1.0 - np.sum(resid ** 2) / syy) if syy > 0 else 1.0
    return slope, r2


def run_scaling(series, tau0, tau_end, window=0.5):
    """Scaling quantities of one run from its list of observables dicts."""
    t_lo = tau0 + window * (tau_end - tau0)
    rows = [o for o in series if o["tau"] >= t_lo - 1e-9 and math.isfinite(o["xi_L"]) and math.isfinite(o["xi_W"])]
    if len(rows) < 3:
        inw = [o for o in series if o["tau"] >= t_lo - 1e-9]
        raise ValueError("%d diagnostics in the scaling window tau >= %g, %d with finite xi_L and xi_W "
                         "(%d recorded, last tau %g)" % (len(inw), t_lo, len(rows), len(series),
                                                          series[-1]["tau"] if series else float("nan")))
    t = [o["tau"] for o in rows]
    sl, r2l = fit_slope(t, [o["xi_L"] for o in rows])
    sw, r2w = fit_slope(t, [o["xi_W"] for o in rows])
    return {"xi_dot_L": sl, "xi_dot_W": sw, "r2_L": r2l, "r2_W": r2w,
            "v2_V": float(np.mean([o["v2_V"] for o in rows])),
            "v2_L": float(np.mean([o["v2_L"] for o in rows])),
            "v2_w": float(np.mean([o["v2_omega"] for o in rows])),
            "points": len(rows)}


def case_configs(ah, name, N, seeds, diag_every, seed0=1):
    era, s, switch = CASES[name]
    cfgs = []
    for k in range(seeds):
        c = ah.config(N, era=era, s=s, seed=seed0 + k, diag_every=diag_every)
        if switch is not None:
            c.tau_ref = switch * c.tau_end
            c.flags |= ah.AH_FLAG_CORE_GROWTH
        cfgs.append(c)
    return cfgs


def scaling_ensemble(N=512, seeds=5, cases=tuple(CASES), diag_every=10, window=0.5, two_step=True):
    """Run every case for `seeds` seeds (one batched job per case; with two_step,
    AH_BATCH_TWO_STEP: lattices of side >= 512 two leapfrog steps per launch) and
    return the per-run and per-case scaling quantities."""
    import paper_1809_00995_gb300 as ah
    out = {"N": N, "seeds": seeds, "diag_every": diag_every, "window": window, "two_step": two_step, "cases": {}}
    for name in cases:
        cfgs = case_configs(ah, name, N, seeds, diag_every)
        t0 = time.perf_counter()
        nsteps = max(int(round((c.tau_end - c.tau0) / c.dt)) for c in cfgs)
        series, stats = ah.ah_batch_run(cfgs, flags=ah.AH_BATCH_TWO_STEP if two_step else 0,
                                        series_cap=nsteps // diag_every + 2)
        wall = time.perf_counter() - t0
        try:
            runs = [run_scaling(ser, c.tau0, c.tau_end, window) for ser, c in zip(series, cfgs)]
        except ValueError as e:
            raise ValueError("%s: %s" % (name, e)) from None
        summary = {}
        for key in ("xi_dot_L", "xi_dot_W", "v2_V", "v2_L", "v2_w"):
            v = np.array([r[key] for r in runs])
            summary[key] = {"mean": float(v.mean()), "std": float(v.std(ddof=1)) if len(v) > 1 else 0.0}
        out["cases"][name] = {"runs": runs, "summary": summary, "seconds": wall,
                              "site_updates_per_s": stats["site_updates"] / stats["seconds"],
                              "tau_ref": cfgs[0].tau_ref, "tau_end": cfgs[0].tau_end,
                              "steps": len(series[0]) and series[0][-1]["step"]}
    return out


def table(res):
    lines = ["| case | xi_dot_L | xi_dot_W | <v^2>_V | <v^2>_L | <v^2>_w |", "|---|---|---|---|---|---|"]
    for name, c in res["cases"].items():
        s = c["summary"]
        cells = ["%.3f +- %.3f" % (s[k]["mean"], s[k]["std"]) for k in ("xi_dot_L", "xi_dot_W", "v2_V", "v2_L", "v2_w")]
        lines.append("| %s | %s |" % (name, " | ".join(cells)))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--diag-every", type=int, default=10)
    ap.add_argument("--window", type=float, default=0.5)
    ap.add_argument("--cases", default=",".join(CASES))
    ap.add_argument("--json", default=None, help="write the full result here")
    ap.add_argument("--one-step", action="store_true", help="one leapfrog step per launch for every lattice")
    a = ap.parse_args()
    res = scaling_ensemble(a.N, a.seeds, tuple(a.cases.split(",")), a.diag_every, a.window, not a.one_step)
    print(table(res))
    for name, c in res["cases"].items():
        print("%s: %d runs, %.1f s, %.3g site-updates/s, tau_ref %.3g, tau_end %.3g"
              % (name, len(c["runs"]), c["seconds"], c["site_updates_per_s"], c["tau_ref"], c["tau_end"]))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
