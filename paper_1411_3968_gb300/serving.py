"""Serving replay: slices of several detectors arrive as Poisson processes
and go through the native engine (trig_submit_slice / trig_poll), which
batches whatever is pending continuously.  Reports slice latency
percentiles against the 200 ms real-time budget of a slice ("Results and
perspectives": a TGPU must keep up with 1 s of data per second).

The request loop and the pollers are Python threads; every call they make
releases the GIL inside libtrig.so, where copies, batching and kernels run.

    python -m paper_1411_3968_gb300.serving --rate 4 --detector-seconds 600
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np

from . import _lib


def warm_up(dets, pools, rounds: int = 2) -> None:
    """Runs every pool slice through the engine a few times, unmeasured: a
    server that runs continuously has its staging memory, device arenas and
    CUDA graphs in place; this brings a fresh process to that state."""
    for _ in range(rounds):
        for i, det in enumerate(dets):
            for t0, st in pools[i]:
                _lib.trig_submit_slice(det, t0, st.hits, st.pmt_off)
        for i, det in enumerate(dets):
            for _ in pools[i]:
                r = _lib.trig_poll(det, 120_000)
                if r is None or r.status != 0:
                    raise RuntimeError(f"warm-up slice failed: {None if r is None else (r.status, r.flags)}")


def replay(dets, pools, rate_factor: float, detector_seconds: float, slice_ns: int, seed: int = 0,
           mode: int = 1, warmup_rounds: int = 2) -> dict:
    """dets[i] receives pools[i][k % len(pools[i])] as its k-th slice; the
    arrival gaps of each detector are exponential with mean
    slice_ns / rate_factor (wall clock)."""
    _lib.trig_engine_set_mode(mode)
    if warmup_rounds:
        warm_up(dets, pools, warmup_rounds)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_per = max(1, int(round(detector_seconds * 1e9 / slice_ns)))
    mean_gap = slice_ns * 1e-9 / rate_factor
    events = []
    for i in range(len(dets)):
        t = 0.0
        for k in range(n_per):
            t += rng.exponential(mean_gap)
            events.append((t, i, k))
    events.sort()
    arrivals = {i: [0.0] * n_per for i in range(len(dets))}
    results = {i: [None] * n_per for i in range(len(dets))}
    received = {i: [0.0] * n_per for i in range(len(dets))}
    errors = []

    def poller(i):
        for k in range(n_per):
            r = _lib.trig_poll(dets[i], 120_000)
            received[i][k] = time.perf_counter()
            if r is None:
                errors.append(f"detector {i}: poll timed out")
                return
            results[i][k] = (r.status, r.latency_ns, r.n_hits, len(r.triggers))

    threads = [threading.Thread(target=poller, args=(i,), daemon=True) for i in range(len(dets))]
    for th in threads:
        th.start()
    t_start = time.perf_counter()
    deferred = 0
    for (t, i, k) in events:
        now = time.perf_counter() - t_start
        if t > now:
            time.sleep(t - now)
        t0, st = pools[i][k % len(pools[i])]
        arrivals[i][k] = t_start + t
        while True:
            try:
                _lib.trig_submit_slice(dets[i], t0, st.hits, st.pmt_off)
                break
            except _lib.TrigError as e:
                if e.code != _lib.TRIG_EAGAIN:
                    raise
                deferred += 1
                time.sleep(0.0005)
    for th in threads:
        th.join()
    t_end = time.perf_counter()
    lat_engine, lat_e2e, per_det = [], [], []
    hits = 0
    bad = 0
    for i in range(len(dets)):
        le = []
        for k in range(n_per):
            r = results[i][k]
            if r is None:
                continue
            status, lat_ns, n_hits, _ = r
            bad += status != 0
            hits += n_hits
            lat_engine.append(lat_ns * 1e-6)
            le.append((received[i][k] - arrivals[i][k]) * 1e3)
        lat_e2e += le
        per_det.append({"n_pmt": int(dets[i].n_pmt), "p50_ms": _pct(le, 50), "p99_ms": _pct(le, 99),
                        "p999_ms": _pct(le, 99.9), "slices": len(le)})
    wall = t_end - t_start
    return {
        "rate_factor": rate_factor,
        "detector_seconds": detector_seconds,
        "slices": int(sum(len(x) for x in results.values())),
        "bad_status": int(bad),
        "errors": errors,
        "wall_s": wall,
        "hits_per_s": hits / wall if wall > 0 else 0.0,
        "p50_ms": _pct(lat_e2e, 50),
        "p99_ms": _pct(lat_e2e, 99),
        "p999_ms": _pct(lat_e2e, 99.9),
        "engine_p99_ms": _pct(lat_engine, 99),
        "budget_ms": slice_ns * 1e-6,
        "deferred_submits": deferred,
        "per_detector": per_det,
    }


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else float("nan")


def main():
    import workload

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--rate", type=float, default=1.0, help="arrival rate in units of real time")
    ap.add_argument("--detector-seconds", type=float, default=20.0)
    ap.add_argument("--pool", type=int, default=4, help="pre-generated slices per detector")
    ap.add_argument("--mode", type=int, default=1, help="0 plain per-slice launches, 1 continuous batching")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    par = dict(workload.DEFAULT_PARAMS)
    wl = workload.cfg_serving_pool(seed=args.seed, slices_per_det=args.pool)
    dets = [_lib.Detector(g.xyz_mm, g.floor_id, par) for g in wl.detectors]
    # the slice pools sit in page-locked host memory, as a DAQ front end's buffers would
    pools = [[(s.t0, workload.Stream(_lib.pinned_copy(s.stream.hits), _lib.pinned_copy(s.stream.pmt_off)))
              for s in wl.submissions if s.det_index == i] for i in range(len(dets))]
    out = replay(dets, pools, args.rate, args.detector_seconds, par["slice_ns"], args.seed, args.mode)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
