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

import paper_1809_00995_gb300 as ah

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
