"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Fields after 20 steps must agree per component within
max|f_gpu - f_ref| / max(max|f_ref|, 1) <= 1e-12 (FP64 state) and 1e-5 (FP32
state); diagnostic sums agree to FP64 rounding and winding counts exactly when
both sides evaluate the same snapshot.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah
from inputs import bps_string, random_state, straight_strings

pytestmark = pytest.mark.gpu

TOL = {ah.AH_FP64: 1e-12, ah.AH_FP32: 1e-5}
KERNELS = [ah.AH_KERNEL_PLAIN, ah.AH_KERNEL_FUSED]


def rel_err(got, ref):
    """Per-component max |got - ref| / max(max |ref|, 1)."""
    return [float(np.max(np.abs(got[c] - ref[c])) / max(np.max(np.abs(ref[c])), 1.0)) for c in range(10)]


def oparams(N, era=ah.AH_RADIATION, s=0.0, seed=1, **kw):
    return O.Params(N=N, era=era, s=s, seed=seed, **kw)


def sim(N, precision, kernel, era=ah.AH_RADIATION, s=0.0, seed=1, **kw):
    return ah.Sim(N, precision=precision, kernel=kernel, era=era, s=s, seed=seed, **kw)


# Tolerances of the diagnostic sums against the oracle on the same snapshot:
# |got - ref| <= rtol |ref| + stol * scale, scale = sum rho (first-order sums) or
# (sum rho)^2 / n_sites (products).  Per-site values are FP64 for an FP64 state
# (rounding only) and FP32 for an FP32 state (relative error of a few 1e-7 per
# site, compensated FP32 accumulation per thread, FP64 across threads).
OBS_TOL = {ah.AH_FP64: (1e-10, 1e-12), ah.AH_FP32: (1e-5, 2e-6)}


def derived_bounds(oo, precision):
    """Bounds on the derived observables (Eqs. defXiV2, defR, defEoS) that the
    sums' tolerances imply, to first order: a sum S is within
    |dS| = rtol |S| + stol * scale of the oracle's, so
      xi_L = sqrt(-mu / mean L):        d xi / xi = |dS_L| / (2 |S_L|),
      R = A / B:                         |dR| = (|dA| + |R| |dB|) / |B|,
      <v^2> = 2 R / (1 + R):             d <v^2> = 2 dR / (1 + R)^2,
      <v^2>_omega = (1 + 3 pL / rhoL)/2: d = 1.5 d(pL / rhoL)."""
    rtol, stol = OBS_TOL[precision]
    S1 = abs(oo["sum_rho"])
    S2 = S1 * S1 / oo["n_sites"]

    def d(name, scale):
        return rtol * abs(oo[name]) + stol * scale

    def ratio(a, b):
        A, B = oo[a], oo[b]
        return (d(a, S2) + abs(A / B) * d(b, S2)) / abs(B)

    out = {"xi_L": abs(oo["xi_L"]) * d("sum_L", S1) / (2 * abs(oo["sum_L"]))}
    for key, (a, b) in {"v2_V": ("sum_KV", "sum_G2V"), "v2_L": ("sum_KL", "sum_G2L")}.items():
        R = oo[a] / oo[b]
        out[key] = 2 * ratio(a, b) / (1 + R) ** 2
    out["v2_omega"] = 1.5 * ratio("sum_pL", "sum_rhoL")
    return out


def compare_obs(go, oo, precision=ah.AH_FP64, exact_windings=True):
    rtol, stol = OBS_TOL[precision]
    S1 = abs(oo["sum_rho"])
    S2 = S1 * S1 / oo["n_sites"]
    names1 = ["L", "rho", "p", "K", "G2", "V", "Eel", "B"]
    okeys = ["sum_L", "sum_rho", "sum_p", "sum_K", "sum_G2", "sum_V", "sum_Eel", "sum_B",
             "sum_KV", "sum_G2V", "sum_KL", "sum_G2L", "sum_pL", "sum_rhoL"]
    for k, name in enumerate(okeys):
        ref, got = oo[name], go["sums"][k]
        scale = S1 if k < len(names1) else S2
        assert abs(got - ref) <= rtol * abs(ref) + stol * scale, (name, got, ref)
    assert abs(go["gauss_max"] - oo["max_gauss"]) <= 1e-12 * max(1.0, oo["max_gauss"]) + 1e-15
    if exact_windings:
        assert list(go["wind_abs_plane"]) == list(oo["sum_abs_W_plane"])
        assert list(go["wind_plane"]) == list(oo["sum_W_plane"])
        assert go["n_pierced"] == oo["n_pierced"]
    assert go["nonfinite"] == 0 and oo["nonfinite"] == 0
    assert abs(go["max_abs_theta"] - oo["max_abs_theta"]) <= 1e-12 * max(1.0, oo["max_abs_theta"])


# ------------------------------------------------------------------ init
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
@pytest.mark.parametrize("N", [4, 7, 32, 64])
def test_initial_state_matches_oracle(N, precision):
    """FP64 state: the oracle's FP64 values to rounding.  FP32 state (phi from
    double-float arithmetic, within 1e-14 of the exact value): the oracle's values
    rounded to FP32, except at most one ulp at a fraction below 1e-4 of the values
    (about 6e-7 expected: values within ~1e-14 of a rounding boundary)."""
    with sim(N, precision, ah.AH_KERNEL_FUSED, seed=77) as s:
        got = s.fields()
    ref = O.init(oparams(N, seed=77))
    if precision == ah.AH_FP64:
        assert np.max(np.abs(got - ref)) < 4e-16
    else:
        r32 = ref.astype(np.float32).astype(np.float64)
        d = np.abs(got - r32)
        ulp = np.spacing(np.abs(r32).astype(np.float32)).astype(np.float64)
        assert np.all(d <= np.maximum(ulp, 2e-16))     # one ulp (or an exact zero against ~1e-16)
        assert np.mean(d > 2e-16) < 1e-4
        assert np.max(np.abs(np.hypot(got[0], got[1]) - 1.0)) < 2e-7
    assert not np.any(got[2:])


# ------------------------------------------------------------------ fields after 20 steps
CASES = [(4, ah.AH_RADIATION, 0.0), (6, ah.AH_MATTER, 1.0), (8, ah.AH_MINKOWSKI, 0.0),
         (33, ah.AH_RADIATION, 0.0), (40, ah.AH_MATTER, 1.0), (17, ah.AH_RADIATION, -0.5)]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
@pytest.mark.parametrize("N,era,s", CASES)
def test_fields_after_20_steps(N, era, s, precision, kernel):
    p = oparams(N, era, s, seed=N + 3)
    with sim(N, precision, kernel, era, s, seed=N + 3) as g:
        f0 = g.fields()                         # the GPU's own initial snapshot
        g.step(20)
        got = g.fields()
        assert g.n == 20
    ref = O.evolve(p, f0.copy(), 0, 20)
    err = rel_err(got, ref)
    assert max(err) <= TOL[precision], err


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_fields_from_random_state(precision, kernel):
    """Random phi, Pi, theta, E: every term of both kicks active from the first step."""
    N = 24
    p = oparams(N, ah.AH_MATTER, 0.5, tau_ref=9.0)
    f = random_state(N, 5)
    with sim(N, precision, kernel, ah.AH_MATTER, 0.5, tau_ref=9.0) as g:
        g.set_fields(f, step=3)
        f0 = g.fields()
        g.step(20)
        got = g.fields()
    ref = O.evolve(p, f0.copy(), 3, 20)
    assert max(rel_err(got, ref)) <= TOL[precision]


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_every_fused_shape_matches_oracle(precision):
    """Every compile-time shape of the fused step (tile height, occupancy, z chunk)
    gives the oracle's fields, on a ragged lattice that spans several tiles."""
    nv = ah.ah_variant_count(precision)
    assert nv >= 2
    tested = set()
    for N in (37, 64):       # ragged tiles; whole 32-site tiles (the TMA-fed shapes need N % 32 == 0)
        p = oparams(N, ah.AH_MATTER, 1.0, seed=21)
        for v in range(nv):
            with sim(N, precision, ah.AH_KERNEL_FUSED, ah.AH_MATTER, 1.0, seed=21) as g:
                try:
                    g.set_variant(v)
                except ah.AhError as e:
                    assert e.status == ah.AH_ERR_ARG and N % 32 != 0
                    continue
                assert g.info["variant"] == v
                f0 = g.fields()
                g.step(20)
                got = g.fields()
                g.sync()
            ref = O.evolve(p, f0.copy(), 0, 20)
            assert max(rel_err(got, ref)) <= TOL[precision], (N, v, max(rel_err(got, ref)))
            tested.add(v)
    assert tested == set(range(nv))


def test_autotune_restores_initial_state_and_picks_a_shape():
    with sim(40, ah.AH_FP32, ah.AH_KERNEL_FUSED, seed=5) as a, sim(40, ah.AH_FP32, ah.AH_KERNEL_FUSED, seed=5) as b:
        f0 = a.fields()
        v = a.autotune(2)
        assert 0 <= v < ah.ah_variant_count(ah.AH_FP32)
        assert np.array_equal(a.fields(), f0) and a.n == 0
        a.step(5)
        with pytest.raises(ah.AhError) as e:
            a.autotune(2)
        assert e.value.status == ah.AH_ERR_BUSY
        b.set_variant(v)
        b.step(5)
        assert np.array_equal(a.fields(), b.fields())
    with sim(40, ah.AH_FP32, ah.AH_KERNEL_FUSED, seed=5, flags=ah.AH_FLAG_AUTOTUNE) as c:
        assert c.info["variant"] == v          # cached per (device, N, precision)


def test_plain_and_fused_agree_fp64():
    with sim(32, ah.AH_FP64, ah.AH_KERNEL_PLAIN, seed=9) as a, sim(32, ah.AH_FP64, ah.AH_KERNEL_FUSED, seed=9) as b:
        a.step(30)
        b.step(30)
        assert max(rel_err(a.fields(), b.fields())) < 1e-13


# ------------------------------------------------------------------ diagnostics
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
@pytest.mark.parametrize("N,era,s", [(32, ah.AH_RADIATION, 0.0), (21, ah.AH_MATTER, 1.0)])
def test_observables_match_oracle_on_same_snapshot(N, era, s, precision):
    p = oparams(N, era, s, seed=4)
    with sim(N, precision, ah.AH_KERNEL_FUSED, era, s, seed=4) as g:
        for n in (0, 10, 20):
            if n:
                g.step(10)
            snap = g.fields()
            go = g.observables()
            oo = O.observables(p, snap, n)
            compare_obs(go, oo, precision)
            assert go["step"] == n and math.isclose(go["tau"], 1.0 + 0.1 * n)
            # each derived observable within the bound its sums' tolerances imply
            bounds = derived_bounds(oo, precision)
            for k, b in bounds.items():
                if math.isfinite(oo[k]) and math.isfinite(b):
                    assert abs(go[k] - oo[k]) <= b + 1e-15, (k, go[k], oo[k], b)
            if n:
                assert go["sum_abs_W"] > 0
                assert abs(go["xi_W"] - oo["xi_W"]) <= 1e-12 * oo["xi_W"]


def test_observables_box_matches_oracle_window():
    N = 24
    p = oparams(N, ah.AH_RADIATION, 0.0, seed=12)
    with sim(N, ah.AH_FP64, ah.AH_KERNEL_FUSED, seed=12) as g:
        g.step(15)
        snap = g.fields()
        for box in [(20, 3, 17, 9, 24, 11), (0, 0, 0, 5, 5, 5), (23, 23, 23, 1, 2, 3)]:
            go = g.observables_box(*box)
            oo = O.observables(p, snap, 15, box=box)
            compare_obs(go, oo, ah.AH_FP64)
            assert go["n_sites"] == box[3] * box[4] * box[5]


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_gauss_law_preserved_on_gpu(precision):
    tol = 1e-12 if precision == ah.AH_FP64 else 2e-4
    with sim(48, precision, ah.AH_KERNEL_FUSED, ah.AH_MATTER, 1.0, seed=5) as g:
        assert g.observables()["gauss_max"] == 0.0
        g.step(100)
        o = g.observables()
    assert o["gauss_max"] < tol and o["sums"][3] > 1.0


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_straight_string_windings_on_gpu(axis):
    N = 20
    f = straight_strings(N, axis=axis)
    with sim(N, ah.AH_FP64, ah.AH_KERNEL_FUSED) as g:
        g.set_fields(f)
        o = g.observables()
    plane = {2: 0, 1: 1, 0: 2}[axis]
    assert o["wind_abs_plane"][plane] == 4 * N and o["wind_plane"][plane] == 0
    assert o["sum_abs_W"] == 4 * N and o["n_pierced"] == 4 * N


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_bps_string_xi_L_on_gpu(precision):
    """The GPU's xi_L = sqrt(-2 pi sigma^2 / mean L) (Eq. defXiV2) on a static
    Bogomolny string in a 16^3 box at spacing 1/4: equal to the oracle's on the
    same snapshot, and within the O(dx^2) lattice error of the box side (one
    string of length N dx in a volume (N dx)^3; the oracle pin measures
    1.46e-3 at this spacing); one pierced plaquette per lattice spacing."""
    N, dx = 64, 0.25
    f = bps_string(N, dx)
    with sim(N, precision, ah.AH_KERNEL_FUSED, ah.AH_MINKOWSKI, 0.0, seed=1, dx=dx, dt=dx / 4) as g:
        g.set_fields(f, 0)
        snap = g.fields()
        go = g.observables()
    p = oparams(N, ah.AH_MINKOWSKI, 0.0, seed=1, dx=dx, dt=dx / 4)
    oo = O.observables(p, snap, 0)
    err = go["xi_L"] / (N * dx) - 1.0
    assert 1.2e-3 < err < 1.7e-3, err
    assert abs(go["xi_L"] - oo["xi_L"]) <= (1e-10 if precision == ah.AH_FP64 else 1e-5) * oo["xi_L"]
    assert go["sum_abs_W"] == N and go["n_pierced"] == N and list(go["wind_abs_plane"]) == [N, 0, 0]


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_exact_diagnostics_flag_matches_oracle(precision):
    N = 20
    p = oparams(N, ah.AH_MATTER, 1.0, seed=6)
    with sim(N, precision, ah.AH_KERNEL_FUSED, ah.AH_MATTER, 1.0, seed=6, flags=ah.AH_FLAG_EXACT_DIAG) as g:
        g.step(12)
        snap = g.fields()
        compare_obs(g.observables(), O.observables(p, snap, 12), ah.AH_FP64)


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
@pytest.mark.parametrize("kind", ["random", "large_theta", "real_fields", "strings", "tiny_phi"])
def test_windings_bit_exact_on_hard_snapshots(precision, kind):
    """Windings of the fast path equal the FP64 arctangent formula on snapshots
    with many plaquettes at or near a branch cut: random fields, link phases far
    outside (-pi, pi], real fields with zero links (edge products exactly on the
    real axis), analytic strings, and fields of magnitude 1e-5."""
    N = 16
    if kind == "random":
        f = random_state(N, 31, phi_amp=1.0, th_amp=3.0)
    elif kind == "large_theta":
        f = random_state(N, 32, th_amp=40.0)
    elif kind == "real_fields":
        f = random_state(N, 33)
        f[1] = 0.0
        f[4:7] = 0.0
    elif kind == "strings":
        f = straight_strings(N, axis=1, x0=0.5, y0=0.25)
    else:                           # |phi| ~ 1e-5: products of four edge values would underflow FP32
        f = random_state(N, 34, th_amp=2.0)
        f[0:2] *= 1e-5
    with sim(N, precision, ah.AH_KERNEL_FUSED) as g:
        g.set_fields(f)
        snap = g.fields()
        go = g.observables()
    oo = O.observables(oparams(N), snap, 0)
    assert list(go["wind_abs_plane"]) == list(oo["sum_abs_W_plane"])
    assert list(go["wind_plane"]) == list(oo["sum_W_plane"])
    assert go["n_pierced"] == oo["n_pierced"]
    if kind != "real_fields":
        assert oo["sum_abs_W"] > 0


# ------------------------------------------------------------------ edge cases and checkpoint
def test_invalid_and_unstable_configs_are_rejected():
    with pytest.raises(ah.AhError) as e:
        ah.Sim(3)
    assert e.value.status == ah.AH_ERR_ARG
    with pytest.raises(ah.AhError) as e:
        ah.Sim(8, dt=0.4)                     # Courant
    assert e.value.status == ah.AH_ERR_ARG
    with pytest.raises(ah.AhError) as e:      # stiff mass term: a(tau0) = 1, s = 1, lambda0 huge
        ah.Sim(8, lambda0=400.0, s=1.0, era=ah.AH_MATTER, tau_ref=1.0)
    assert e.value.status == ah.AH_ERR_UNSTABLE
    with ah.Sim(8) as g:
        with pytest.raises(ah.AhError):
            g.step(-1)
        g.step(0)
        assert g.n == 0
        with pytest.raises(ah.AhError):
            g.observables_box(0, 0, 0, 9, 1, 1)
    with pytest.raises(ah.AhError):
        ah.ah_create(3, 0.5, 0.1, 1, 0.0, 2.0, 1.0, 1)


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_checkpoint_resume_is_bit_identical(precision):
    with sim(20, precision, ah.AH_KERNEL_FUSED, seed=8) as a:
        a.step(7)
        snap = a.fields()
        a.step(9)
        want = a.fields()
    with sim(20, precision, ah.AH_KERNEL_FUSED, seed=999) as b:
        b.set_fields(snap, step=7)
        b.step(9)
        assert np.array_equal(b.fields(), want)


def test_stepping_is_deterministic():
    outs = []
    for _ in range(2):
        with sim(36, ah.AH_FP32, ah.AH_KERNEL_FUSED, seed=3) as g:
            g.step(25)
            outs.append((g.fields(), g.observables()["sums"]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


# ------------------------------------------------------------------ full-size cases
@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_256cubed_first_20_steps_match_oracle(precision):
    """256^3, radiation era, s = 0, seed 2: all fields of the whole lattice after 20
    steps, the oracle run from the GPU's initial snapshot."""
    N = 256
    p = oparams(N, ah.AH_RADIATION, 0.0, seed=2)
    with sim(N, precision, ah.AH_KERNEL_FUSED, ah.AH_RADIATION, 0.0, seed=2, flags=ah.AH_FLAG_AUTOTUNE) as g:
        f0 = g.fields()
        g.step(20)
        got = g.fields()
        go = g.observables()
    ref = O.evolve(p, f0, 0, 20)
    assert max(rel_err(got, ref)) <= TOL[precision]
    compare_obs(go, O.observables(p, got, 20), precision)
    del ref, got, f0


def test_1024cubed_fp32_light_cone_windows():
    """1024^3 FP32, matter era, s = 1, seed 3, in the bench's launch configuration
    (autotuned shape): after 20 steps the fields in three 16^3 windows (two across
    the periodic seam) equal the oracle's evolution of (16 + 2*20)^3 windows of the
    same initial lattice; diagnostics of sub-boxes match the oracle on fetched
    windows; the Gauss residual stays at FP32 roundoff over the whole lattice."""
    N, k, b = 1024, 20, 16
    p = oparams(N, ah.AH_MATTER, 1.0, seed=3)
    with sim(N, ah.AH_FP32, ah.AH_KERNEL_FUSED, ah.AH_MATTER, 1.0, seed=3, flags=ah.AH_FLAG_AUTOTUNE) as g:
        g.step(k)
        for org in [(1016, 5, 1019), (300, 1010, 7), (511, 512, 640)]:
            M = b + 2 * k
            w0 = [(o - k) % N for o in org]
            win = O.init(p, M=M, origin=w0)
            win32 = win.astype(np.float32).astype(np.float64)      # the FP32 state's initial values
            O.evolve(p, win32, 0, k)
            got = g.fields(*org, b, b, b)
            ref = win32[:, k:k + b, k:k + b, k:k + b]
            assert max(rel_err(got, ref)) <= TOL[ah.AH_FP32], org
            # diagnostics of the b^3 box against the oracle on a (b+2)^3 fetched window
            fw = g.fields(*[(o - 1) % N for o in org], b + 2, b + 2, b + 2)
            go = g.observables_box(*org, b, b, b)
            oo = O.observables(p, fw, k, box=(1, 1, 1, b, b, b))
            compare_obs(go, oo, ah.AH_FP32)
        o = g.observables()
    assert o["n_sites"] == N ** 3 and o["nonfinite"] == 0
    assert o["gauss_rel"] < 1e-5


def test_1300cubed_fp32_64bit_site_indices():
    """The largest lattices (N^3 >= 2^31, up to the ~1660^3 FP32 state that fits
    in HBM) take the 64-bit-index instantiations of the step and of the
    diagnostics pass.  1300^3 FP32 (131 GB), radiation era: windows beyond linear
    index 2^31 and across the seam equal the oracle after 20 steps, and the
    whole-lattice diagnostics equal the site-parallel box kernel on the same
    snapshot (sums to FP64 rounding of FP32 values, windings exactly)."""
    N, k, b = 1300, 20, 12
    assert N ** 3 >= 2 ** 31
    p = oparams(N, ah.AH_RADIATION, 0.0, seed=6)
    with sim(N, ah.AH_FP32, ah.AH_KERNEL_FUSED, ah.AH_RADIATION, 0.0, seed=6, flags=ah.AH_FLAG_AUTOTUNE) as g:
        g.step(k)
        for org in [(1295, 3, 1290), (640, 1297, 1280)]:
            M = b + 2 * k
            win = O.init(p, M=M, origin=[(o - k) % N for o in org])
            win32 = win.astype(np.float32).astype(np.float64)
            O.evolve(p, win32, 0, k)
            got = g.fields(*org, b, b, b)
            assert max(rel_err(got, win32[:, k:k + b, k:k + b, k:k + b])) <= TOL[ah.AH_FP32], org
        whole = g.observables()
        site = g.observables_box(1, 0, 0, N, N, N)      # the same sites, site-parallel kernel
    assert whole["n_sites"] == N ** 3 and whole["nonfinite"] == 0 and whole["n_pierced"] > 0
    assert whole["wind_abs_plane"] == site["wind_abs_plane"] and whole["wind_plane"] == site["wind_plane"]
    assert whole["n_pierced"] == site["n_pierced"]
    S1 = abs(site["sums"][1])
    for kk in range(14):
        scale = S1 if kk < 8 else S1 * S1 / N ** 3
        assert abs(whole["sums"][kk] - site["sums"][kk]) <= 1e-6 * abs(site["sums"][kk]) + 1e-7 * scale, kk
    assert whole["max_abs_theta"] == site["max_abs_theta"]
    assert abs(whole["gauss_max"] - site["gauss_max"]) <= 1e-12 * max(1.0, site["gauss_max"])


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
def test_zero_gradient_denominators_are_reported_not_trapped(precision):
    """Uniform phi with Pi != 0: |D phi|^2 = 0 at every site, so R_V = sum K V /
    sum G2 V divides by zero; the observables carry IEEE inf/NaN for the velocity
    estimators (as the oracle does) and the call still succeeds."""
    N = 8
    f = np.zeros((10, N, N, N))
    f[0], f[1] = 0.6, 0.5                     # uniform phi, |phi|^2 != sigma^2 so V != 0
    f[2], f[3] = 0.3, -0.1                    # uniform Pi
    p = oparams(N, ah.AH_MINKOWSKI)
    with sim(N, precision, ah.AH_KERNEL_FUSED, ah.AH_MINKOWSKI) as g:
        g.set_fields(f, step=0)
        go = g.observables()
    oo = O.observables(p, f, 0)
    assert go["sums"][4] == 0.0 and go["sums"][9] == 0.0          # sum G2, sum G2 V
    assert math.isinf(go["R_V"]) and math.isinf(oo["R_V"])
    assert math.isnan(go["v2_V"]) and math.isnan(oo["v2_V"])
    assert go["nonfinite"] == 0


@pytest.mark.parametrize("precision", [ah.AH_FP64, ah.AH_FP32])
@pytest.mark.parametrize("N", [4, 5, 7])
def test_observables_on_the_smallest_lattices(N, precision):
    """Lattices smaller than one 32 x 8 tile (the tile wraps onto itself, every
    neighbour is a periodic image): whole-lattice diagnostics equal the oracle's
    on the same snapshot, windings exactly."""
    p = oparams(N, ah.AH_RADIATION, 0.0, seed=N)
    f = random_state(N, 50 + N, th_amp=2.0, phi_amp=1.0)
    with sim(N, precision, ah.AH_KERNEL_FUSED, ah.AH_RADIATION, 0.0, seed=N) as g:
        g.set_fields(f, step=5)
        g.step(3)
        snap = g.fields()
        go = g.observables()
    compare_obs(go, O.observables(p, snap, 8), precision)


def test_state_larger_than_hbm_reports_oom_and_the_device_stays_usable():
    """2048^3 FP32 needs 515 GB of state: creation fails with AH_ERR_OOM (a refused
    allocation, no fault) and the next simulation on the device works."""
    with pytest.raises(ah.AhError) as e:
        ah.ah_create_ex(ah.config(2048))
    assert e.value.status == ah.AH_ERR_OOM
    with sim(16, ah.AH_FP32, ah.AH_KERNEL_FUSED) as g:
        g.step(3)
        assert g.observables()["nonfinite"] == 0


def test_two_simulations_from_two_threads_match_sequential_runs():
    """Host-side thread safety: two simulations (different sizes, one autotuned)
    created, stepped and measured from two threads at once give bit for bit the
    fields and observables of the same runs done one after the other."""
    import threading

    def run(N, seed, flags, out, key):
        with sim(N, ah.AH_FP32, ah.AH_KERNEL_FUSED, ah.AH_MATTER, 1.0, seed=seed, flags=flags) as g:
            v = g.info["variant"]
            g.step(15)
            o = g.observables()
            out[key] = (v, g.fields(), o["sums"], o["wind_abs_plane"])

    jobs = [(40, 3, ah.AH_FLAG_AUTOTUNE), (27, 4, 0)]
    seq, par = {}, {}
    for i, (N, seed, fl) in enumerate(jobs):
        run(N, seed, fl, seq, i)
    threads = [threading.Thread(target=run, args=(N, seed, fl, par, i)) for i, (N, seed, fl) in enumerate(jobs)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i in range(len(jobs)):
        vs, fs, ss, ws = seq[i]
        vp, fp, sp, wp = par[i]
        assert vs == vp
        assert np.array_equal(fs, fp) and ss == sp and ws == wp, i
