"""Host logic of the serving replay (no GPU): run specifications and the
breakdown of the engine's per-slice trace into submit, copy wait, queue,
batch and read-back times."""
import numpy as np

from paper_1411_3968_gb300 import _lib
from paper_1411_3968_gb300 import serving


def test_run_specifications_parse():
    assert serving._parse_run("4:1:600") == (4.0, 1, 600.0)
    assert serving._parse_run("0.5:0:30") == (0.5, 0, 30.0)
    assert serving._parse_run("sat:1:20") == ("sat", 1, 20.0)
    assert serving._parse_run("burst:0:4") == ("burst", 0, 4.0)


def _trace(n, rng):
    tr = np.zeros(n, _lib.TRACE_DTYPE)
    t = np.cumsum(rng.integers(1_000_000, 5_000_000, n))           # submissions 1-5 ms apart
    sub = rng.integers(100_000, 3_000_000, n)                        # 0.1-3 ms in trig_submit_slice
    wait = (sub * rng.uniform(0.2, 0.9, n)).astype(np.int64)         # part of it waiting for copies
    queue = rng.integers(10_000, 200_000, n)
    batch = rng.integers(100_000, 3_000_000, n)
    back = rng.integers(20_000, 400_000, n)
    tr["slice_id"] = np.arange(n)
    tr["batch"] = np.arange(n) // 2 + 1
    tr["batch_slices"] = 2
    tr["n_pmt"] = np.where(np.arange(n) % 4 == 3, 2688, 84)
    tr["t_submit_ns"] = t
    tr["t_queued_ns"] = t + sub
    tr["t_launch_ns"] = t + sub + queue
    tr["t_stats_ns"] = t + sub + queue + batch
    tr["t_done_ns"] = t + sub + queue + batch + back
    tr["device_ms"] = batch * 1e-6 * 0.9
    tr["copy_wait_us"] = wait // 1000
    tr["continuation"] = 1
    return tr, sub, wait, queue, batch, back


def test_trace_summary_parts_and_tail():
    rng = np.random.Generator(np.random.PCG64(3))
    tr, sub, wait, queue, batch, back = _trace(2000, rng)
    out = serving.trace_summary(tr)
    for key, ns in (("submit_ms", sub), ("queue_ms", queue), ("batch_ms", batch), ("readback_ms", back),
                    ("total_ms", sub + queue + batch + back)):
        for q, name in ((50, "p50"), (99, "p99"), (99.9, "p999")):
            assert abs(out[key][name] - np.percentile(ns * 1e-6, q)) < 1e-9, (key, name)
    assert abs(out["copy_wait_ms"]["p50"] - np.percentile((wait // 1000) * 1e-3, 50)) < 1e-9
    assert abs(out["device_ms"]["p50"] - np.percentile(tr["device_ms"], 50)) < 1e-6
    assert out["batch_slices"] == {"mean": 2.0, "max": 2}
    assert out["batches"] == 1000
    assert out["continuation_share"] == 1.0
    # the slowest 0.1 %: the slices at or above the 99.9th percentile of the total
    tot = (sub + queue + batch + back) * 1e-6
    slow = tot >= np.percentile(tot, 99.9)
    assert abs(out["slowest"]["total_ms"] - tot[slow].mean()) < 1e-9
    assert out["slowest"]["n_pmt"] == sorted(set(int(x) for x in tr["n_pmt"][slow]))


def test_trace_summary_of_an_empty_trace():
    assert serving.trace_summary(np.zeros(0, _lib.TRACE_DTYPE)) == {}
