"""GPU test of ah_observables_noalloc, the diagnostics entry point that allocates
no device memory.  It serves callers that cannot call cudaMalloc: code inside a
host framework that owns the whole device memory pool through its own
allocator, loops that must not block on the driver's allocator once running,
and sandboxes that forbid new device allocations after start-up.  Its scratch
lives in a fixed static device array, so two calls in a row must both give the
sums of the allocating entry point (ah_observables) on the same state.

Collected last (file name) so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
import paper_1809_00995_gb300 as ah
from inputs import random_state

pytestmark = pytest.mark.gpu

RTOL, STOL = 1e-5, 2e-6      # FP32-state diagnostic tolerance of the parity tests


def _read_sums(t):
    return ah.ah_sums.from_buffer_copy(t.cpu().numpy().tobytes())


def test_noalloc_matches_observables_on_two_calls():
    torch = pytest.importorskip("torch")
    N = 40
    with ah.Sim(N, precision=ah.AH_FP32, era=ah.AH_MATTER, s=1.0, seed=11) as g:
        g.step(25)
        snap = g.fields()                 # exact FP64 copy of the FP32 state
        ref = g.observables()
        cfg, step = g.cfg, g.n
    dev = torch.device("cuda", 0)
    bufs = [torch.from_numpy(np.ascontiguousarray(snap[c], dtype=np.float32).ravel()).to(dev) for c in range(10)]
    out = torch.empty(26, dtype=torch.int64, device=dev)          # one ah_sums (208 bytes)
    stream = torch.cuda.current_stream()
    scale = abs(ref["sums"][1])
    for _ in range(2):
        out.fill_(-1)                     # every field must be overwritten by the call
        ah.ah_observables_noalloc([b.data_ptr() for b in bufs], N, cfg, step, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = _read_sums(out)
        for k in range(16):
            r, x = ref["sums"][k], got.sums[k]
            sc = scale if k < 8 else scale * scale / N ** 3
            assert abs(x - r) <= RTOL * abs(r) + STOL * sc, (k, x, r)
        assert list(got.wind_abs_plane) == list(ref["wind_abs_plane"])
        assert list(got.wind_plane) == list(ref["wind_plane"])
        assert got.n_pierced == ref["n_pierced"] and got.n_pierced > 0
        assert got.nonfinite == 0
        assert abs(got.gauss_max - ref["gauss_max"]) <= 1e-12 * max(1.0, ref["gauss_max"])
        assert got.max_abs_theta == ref["max_abs_theta"]


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    N = 8
    cfg = ah.config(N)
    dev = torch.device("cuda", 0)
    bufs = [torch.zeros(N ** 3, dtype=torch.float32, device=dev) for _ in range(10)]
    out = torch.zeros(26, dtype=torch.int64, device=dev)
    ptrs = [b.data_ptr() for b in bufs]
    for bad_N in (N + 1, 3, 4096):
        with pytest.raises(ah.AhError) as e:
            ah.ah_observables_noalloc(ptrs, bad_N, cfg, 0, out.data_ptr())
        assert e.value.status == ah.AH_ERR_ARG
    cfg64 = ah.config(N, precision=ah.AH_FP64)
    with pytest.raises(ah.AhError) as e:
        ah.ah_observables_noalloc(ptrs, N, cfg64, 0, out.data_ptr())
    assert e.value.status == ah.AH_ERR_ARG


def _sign_state(M, seed):
    """phi = +-1 (random signs, real), theta = 0, random Pi and E: every edge
    product conj(phi^a) e^{i theta} phi^b is exactly +1 or -1, and each -1 lies on
    the branch cut of Arg, so the fast winding path must hand the plaquette on."""
    f = random_state(M, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    f[0] = rng.choice([-1.0, 1.0], size=(M, M, M))
    f[1] = 0.0
    f[4:7] = 0.0
    return f


def _listed_plaquettes(f):
    """Plaquettes of a sign state whose four corners do not all share one sign:
    exactly those with an edge product on the branch cut."""
    s = f[0]
    n = 0
    for ax_i, ax_j in [(2, 1), (2, 0), (1, 0)]:          # (12), (13), (23) in (z, y, x) axes
        a, b = np.roll(s, -1, axis=ax_i), np.roll(s, -1, axis=ax_j)
        c = np.roll(b, -1, axis=ax_i)
        n += int(np.count_nonzero(~((s == a) & (s == b) & (s == c))))
    return n


def _noalloc(torch, fields, N, cfg, step):
    dev = torch.device("cuda", 0)
    bufs = [torch.from_numpy(np.ascontiguousarray(fields[c], dtype=np.float32).ravel()).to(dev) for c in range(10)]
    out = torch.full((26,), -1, dtype=torch.int64, device=dev)
    ah.ah_observables_noalloc([b.data_ptr() for b in bufs], N, cfg, step, out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return _read_sums(out)


def test_noalloc_list_overflow_recounts_windings_in_fp64():
    """More near-cut plaquettes than the static list holds (2^18): the call
    recounts every winding of the lattice in FP64.  On a 64^3 sign state about
    7/8 of the 786432 plaquettes are listed; the windings still equal those of
    ah_observables (whose list holds them all) and of the oracle's arctangent
    formula, the energies those of ah_observables; a second call in a row
    gives the same."""
    torch = pytest.importorskip("torch")
    N = 64
    f = _sign_state(N, 21)
    assert _listed_plaquettes(f) > 2 ** 18
    cfg = ah.config(N, precision=ah.AH_FP32, era=ah.AH_RADIATION, seed=21)
    with ah.Sim(N, precision=ah.AH_FP32, era=ah.AH_RADIATION, seed=21) as g:
        g.set_fields(f, 7)
        snap = g.fields()
        ref = g.observables()
    oo = O.observables(O.Params(N=N, era=O.RADIATION, seed=21), snap, 7)
    assert list(ref["wind_abs_plane"]) == list(oo["sum_abs_W_plane"]) and ref["n_pierced"] == oo["n_pierced"]
    assert ref["n_pierced"] > 0
    scale = abs(ref["sums"][1])
    for _ in range(2):
        got = _noalloc(torch, snap, N, cfg, 7)
        assert list(got.wind_abs_plane) == list(ref["wind_abs_plane"])
        assert list(got.wind_plane) == list(ref["wind_plane"])
        assert got.n_pierced == ref["n_pierced"]
        for k in range(8):
            assert abs(got.sums[k] - ref["sums"][k]) <= RTOL * abs(ref["sums"][k]) + STOL * scale, k
        assert got.nonfinite == 0


def test_noalloc_past_2_31_sites():
    """1296^3 = 2.18e9 sites, past 2^31: 64-bit site indices in every kernel of
    the call.  The lattice is a 16^3 tile repeated 81 times along each axis, so
    every sum is 81^3 times the tile's (FP32 per-site values are identical in each
    copy) and every winding count exactly so.  First a generic random tile,
    then a sign tile whose 81^3 copies of listed plaquettes overflow the list, so
    that the FP64 recount runs over the whole lattice."""
    torch = pytest.importorskip("torch")
    T, R = 16, 81
    N = T * R
    assert N ** 3 > 2 ** 31
    dev = torch.device("cuda", 0)
    bufs = [torch.empty(N ** 3, dtype=torch.float32, device=dev) for _ in range(10)]
    out = torch.empty(26, dtype=torch.int64, device=dev)
    cfg = ah.config(N, precision=ah.AH_FP32, era=ah.AH_MATTER, s=1.0, seed=5)
    cfg_t = ah.config(T, precision=ah.AH_FP32, era=ah.AH_MATTER, s=1.0, seed=5)
    cfg_t.tau_end, cfg_t.tau_ref = cfg.tau_end, cfg.tau_ref          # the same couplings at step 9
    try:
        for tile in (random_state(T, 31), _sign_state(T, 32)):
            with ah.Sim(T, precision=ah.AH_FP32, era=ah.AH_MATTER, s=1.0, seed=5, tau_end=cfg.tau_end,
                        tau_ref=cfg.tau_ref) as g:
                g.set_fields(tile, 9)
                snap = g.fields()
                ref = g.observables()
            for c in range(10):
                t = torch.from_numpy(np.ascontiguousarray(snap[c], dtype=np.float32)).to(dev)
                bufs[c].view(R, T, R, T, R, T).copy_(t[None, :, None, :, None, :].expand(R, T, R, T, R, T))
            out.fill_(-1)
            ah.ah_observables_noalloc([b.data_ptr() for b in bufs], N, cfg, 9, out.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = _read_sums(out)
            m = R ** 3
            assert list(got.wind_abs_plane) == [m * w for w in ref["wind_abs_plane"]]
            assert list(got.wind_plane) == [m * w for w in ref["wind_plane"]]
            assert got.n_pierced == m * ref["n_pierced"] and got.nonfinite == 0
            scale = abs(ref["sums"][1])
            for k in range(16):
                sc = scale if k < 8 else scale * scale / T ** 3
                assert abs(got.sums[k] - m * ref["sums"][k]) <= m * (RTOL * abs(ref["sums"][k]) + STOL * sc), k
            assert got.max_abs_theta == ref["max_abs_theta"]
            assert abs(got.gauss_max - ref["gauss_max"]) <= 1e-12 * max(1.0, ref["gauss_max"])
    finally:
        del bufs
        torch.cuda.empty_cache()
