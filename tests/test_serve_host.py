"""Host-side logic of the solve server (no GPU): accuracy routing, the memory estimate
that admission uses, percentiles, and the seeded Poisson arrivals."""
import types

import numpy as np

from paper_2506_04489_gb300 import serve


def test_accuracy_routing():
    assert serve.precision_for(1e-6) == "fp32"
    assert serve.precision_for(1e-5) == "fp32"
    assert serve.precision_for(1e-12) == "df32"
    assert serve.precision_for(1e-9) == "df32"


def test_entry_bytes_counts_workspace_and_buffers():
    # double-float 256^3, batch 8: workspace 8 * 16 * 256 * 512 * 264 B dominates
    b = serve.entry_bytes(256, "df32", 8)
    work = 8 * 16 * 256 * 512 * 264
    io = 2 * 8 * 256 ** 3 * 8
    assert work + io < b < work + io + 400e6
    assert serve.entry_bytes(256, "fp32", 8) < b
    assert serve.entry_bytes(128, "df32", 8) < b / 6


def test_percentiles_nearest_rank():
    v = list(range(1, 101))
    assert serve.percentile(v, 50) == 50
    assert serve.percentile(v, 99) == 99
    assert serve.percentile([7.0], 99) == 7.0


def test_summarize_window_and_throughput():
    reqs = [types.SimpleNamespace(arrival=t, done_at=t + 0.002 * (1 + i % 3)) for i, t in enumerate(np.arange(0, 1, 0.01))]
    s = serve.summarize(reqs, 0.5, 1.0)
    assert s["requests"] == 50
    assert 2.0 <= s["p50_ms"] <= 6.0 and s["p99_ms"] <= 6.0 + 1e-9
    assert 90 < s["solves_per_s"] < 110


def test_poisson_arrivals_are_seeded():
    # the same seed gives the same sizes, accuracies and inter-arrival gaps
    def draw(seed):
        rng = np.random.Generator(np.random.PCG64(seed))
        out = []
        for _ in range(20):
            out.append((int(rng.integers(6)), int(rng.integers(2)), float(rng.exponential(1 / 200))))
        return out
    assert draw(0) == draw(0) and draw(0) != draw(1)
    gaps = [g for _, _, g in draw(0)]
    assert 0 < np.mean(gaps) < 0.02


def test_batch_cap_by_points():
    # 256^3 grids: two per launch under a 2 x 256^3 point cap; small grids up to max_batch
    assert serve.batch_cap(256, 8, 2 * 256 ** 3) == 2
    assert serve.batch_cap(128, 8, 2 * 256 ** 3) == 8
    assert serve.batch_cap(64, 8, 2 * 256 ** 3) == 8
    # a grid larger than the cap still runs, alone
    assert serve.batch_cap(512, 8, 2 * 256 ** 3) == 1


def test_summarize_per_key():
    Done = serve.Done
    reqs = [Done(0.1 * i, 0.1 * i + (0.001 if i % 2 else 0.004), (32 if i % 2 else 256, "df32")) for i in range(10)]
    s = serve.summarize(reqs, 0.0, 1.0)
    assert set(s["by_key"]) == {"n32_df32", "n256_df32"}
    assert s["by_key"]["n32_df32"]["requests"] == 5
    assert abs(s["by_key"]["n256_df32"]["p99_ms"] - 4.0) < 1e-9


def test_small_batches_take_high_priority_slots():
    # slots 0 and 1 are the high-priority streams
    assert serve.pick_slot([0, 1, 2, 3], 2, small=True) == 0
    assert serve.pick_slot([0, 1, 2, 3], 2, small=False) == 2
    assert serve.pick_slot([1, 3], 2, small=True) == 1
    assert serve.pick_slot([0, 1], 2, small=False) == 0  # no normal slot free: take any
    assert serve.pick_slot([2], 2, small=True) == 2


def test_native_memory_estimate_matches_the_host_one():
    # the library's admission estimate (sp_server_entry_bytes) is the one documented here
    from paper_2506_04489_gb300 import build
    build.build()
    from paper_2506_04489_gb300 import _native as N
    for mb in (1, 8):
        cfg = N.ServerConfig(-1.0, 1.0, 1e9, mb, 4, 2, 2, 2 * 128 ** 3, 256 ** 3)
        for n in (32, 96, 128, 256):
            for prec, code in (("fp32", 1), ("df32", 3)):
                assert N.lib.sp_server_entry_bytes(cfg, n, code) == serve.entry_bytes(n, prec, mb)
