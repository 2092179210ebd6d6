"""Host-side logic of bench.py (no GPU): the choice of the two-step mode and the
lookup of the committed DRAM-traffic records."""
import json

import pytest

import bench


def test_two_step_mode_rule():
    assert bench.use_two_step(0, 50)                  # FP32, even diagnostics interval
    assert not bench.use_two_step(0, 5)               # odd interval: not a whole number of pairs
    assert not bench.use_two_step(1, 20)              # FP64 has no two-step kernel
    assert not bench.use_two_step(0, 50, single_step=True)


def test_traffic_records_match_their_kernel_sources():
    """Every committed record names a shape and the lattice it was captured on,
    which holds a few GB at most (ncu saves and restores device memory between
    its passes); while it was taken on the kernel sources as they are now the
    bench reports it, scaled to its own lattice by the site count (after a
    kernel change the bench reports no traffic until the kernel is captured
    again)."""
    with open(bench.TRAFFIC_FILE) as f:
        recs = json.load(f)
    assert set(recs) == {"k_fused", "k_fused2"}
    for kernel, r in recs.items():
        assert r["N"] ** 3 * 80 <= 8e9                 # the captured state: 80 B/site at most
        if r["sources_sha256_16"] != bench.kernel_source_hash(kernel):
            assert bench.traffic_per_launch(1024, kernel, r["variant"]) is None
            continue
        for N in (r["N"], 1024):
            got = bench.traffic_per_launch(N, kernel, r["variant"])
            assert got == pytest.approx(r["dram_bytes_per_site"] * N ** 3)
        # a bit above the algorithmic 80 B per site and launch (one read and one
        # write of the FP32 state), never below it by more than the counters' noise
        assert 79.0 <= r["dram_bytes_per_site"] < 100.0


def test_traffic_lookup_refuses_other_shapes_and_kernels():
    with open(bench.TRAFFIC_FILE) as f:
        r = json.load(f)["k_fused2"]
    assert bench.traffic_per_launch(1024, "k_fused2", "no_such_shape") is None
    assert bench.traffic_per_launch(1024, "k_fused", r["variant"]) is None
