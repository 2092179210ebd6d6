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
    """Every committed record names a shape and a size; while it was taken on the
    kernel sources as they are now the bench reports it (after a kernel change the
    bench reports no traffic until the kernel is captured again)."""
    with open(bench.TRAFFIC_FILE) as f:
        recs = json.load(f)
    assert set(recs) == {"k_fused", "k_fused2"}
    for kernel, r in recs.items():
        if r["sources_sha256_16"] != bench.kernel_source_hash(kernel):
            assert bench.traffic_per_launch(r["N"], kernel, r["variant"]) is None
            continue
        got = bench.traffic_per_launch(r["N"], kernel, r["variant"])
        assert got == pytest.approx(r["dram_bytes_per_site"] * r["N"] ** 3)
        # a bit above the algorithmic 80 B per site and launch (one read and one
        # write of the FP32 state), never below it
        assert 80.0 <= r["dram_bytes_per_site"] < 100.0


def test_traffic_lookup_refuses_other_shapes_and_sizes():
    with open(bench.TRAFFIC_FILE) as f:
        r = json.load(f)["k_fused2"]
    assert bench.traffic_per_launch(r["N"] // 2, "k_fused2", r["variant"]) is None
    assert bench.traffic_per_launch(r["N"], "k_fused2", "no_such_shape") is None
    assert bench.traffic_per_launch(r["N"], "k_fused", r["variant"]) is None
