"""Scaling-ensemble analysis (Table 3 quantities): the fits on exact synthetic
series (CPU) and a small batched ensemble end to end (GPU)."""
import math

import numpy as np
import pytest

from paper_1809_00995_gb300 import ensemble as E


def test_fit_slope_is_exact_on_a_line_and_reports_r2():
    t = np.linspace(10, 20, 11)
    s, r2 = E.fit_slope(t, 0.31 * t + 2.5)
    assert abs(s - 0.31) < 1e-14 and abs(r2 - 1.0) < 1e-14
    s, r2 = E.fit_slope(t, 0.31 * t + np.sin(7 * t))
    assert abs(s - 0.31) < 0.1 and r2 < 1.0


def test_run_scaling_uses_the_second_half_of_the_run():
    tau0, tau_end = 1.0, 33.0
    ser = []
    for k in range(33):
        tau = tau0 + k
        early = tau < 17.0                      # a different slope before the window
        ser.append({"tau": tau, "xi_L": (2.0 * tau if early else 0.3 * tau + 29.2),
                    "xi_W": 0.28 * tau, "v2_V": 0.34, "v2_L": 0.31 if not early else 9.0,
                    "v2_omega": 0.32})
    ser[0]["xi_L"] = math.nan                   # xi_L undefined while mean L > 0
    r = E.run_scaling(ser, tau0, tau_end)
    assert r["points"] == 17
    assert abs(r["xi_dot_L"] - 0.3) < 1e-12 and abs(r["xi_dot_W"] - 0.28) < 1e-12
    assert r["v2_L"] == pytest.approx(0.31) and r["v2_w"] == pytest.approx(0.32)


@pytest.mark.gpu
def test_small_ensemble_runs_end_to_end():
    res = E.scaling_ensemble(N=48, seeds=2, cases=("radiation_s0", "radiation_s1"), diag_every=4)
    for name, c in res["cases"].items():
        assert len(c["runs"]) == 2
        for r in c["runs"]:
            assert r["points"] >= 10
            for k in ("xi_dot_L", "xi_dot_W", "v2_V", "v2_L", "v2_w"):
                assert math.isfinite(r[k]), (name, k)
            assert r["xi_dot_W"] > 0                   # the network dilutes
        assert c["tau_end"] == 12.0
    assert res["cases"]["radiation_s1"]["tau_ref"] == pytest.approx(6.0)
