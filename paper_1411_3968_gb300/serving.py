"""Serving replay: slices of several detectors arrive as Poisson processes
and go through the native engine (trig_submit_slice / trig_poll), which
batches whatever is pending continuously.  Reports slice latency
percentiles against the 200 ms real-time budget of a slice ("Results and
perspectives": a TGPU must keep up with 1 s of data per second), the
served hits/s, and where the latency goes (the engine's per-slice trace).

Each detector replays a pool of contiguous slices: the pool's first slice
carries both halos, every later one starts at its t0 and takes its leading
halo from the previous slice's tail that the engine keeps on the device
(is_continuation = 1).  A run is rate:mode:detector_seconds, where rate is
the arrival rate in units of real time (or "sat": every slice submitted at
once, which measures capacity through the submitting thread's copies; or
"burst": every slice submitted while the engine holds its launches, then
released at once, which measures the device side's capacity with the
copies already done) and mode is the engine's (0 plain per-slice launches,
1 continuous batching).

Each detector has a submitting thread and a polling thread (Python
threads; every call they make releases the GIL inside libtrig.so, where
copies, batching and kernels run).

    python -m paper_1411_3968_gb300.serving --pool 20 --runs 4:1:600 4:0:600 1:1:600 1:0:600 \
        sat:1:60 sat:0:60 burst:1:4 burst:0:4
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np

from . import _lib


def warm_up(dets, pools, rounds: int = 1) -> None:
    """Runs every pool slice through the engine, unmeasured: a server that
    runs continuously has its staging memory and device arenas in place;
    this brings a fresh process to that state."""
    for _ in range(rounds):
        for i, det in enumerate(dets):
            for (t0, st, cont) in pools[i]:
                _submit(det, t0, st, cont)
        for i, det in enumerate(dets):
            for _ in pools[i]:
                r = _lib.trig_poll(det, 120_000)
                if r is None or r.status != 0:
                    raise RuntimeError(f"warm-up slice failed: {None if r is None else (r.status, r.flags)}")


def _submit(det, t0, st, cont) -> int:
    deferred = 0
    while True:
        try:
            _lib.trig_submit_slice(det, t0, st.hits, st.pmt_off, is_continuation=cont)
            return deferred
        except _lib.TrigError as e:
            if e.code != _lib.TRIG_EAGAIN:
                raise
            deferred += 1
            time.sleep(0.0005)


def replay(dets, pools, rate_factor, detector_seconds: float, slice_ns: int, seed: int = 0, mode: int = 1,
           warmup_rounds: int = 1, trace_out: str | None = None) -> dict:
    """dets[i] receives pools[i][k % len(pools[i])] as its k-th slice; the
    arrival gaps of each detector are exponential with mean
    slice_ns / rate_factor (wall clock), or zero for rate_factor "sat"."""
    _lib.trig_engine_set_mode(mode)
    if warmup_rounds:
        warm_up(dets, pools, warmup_rounds)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_per = max(1, int(round(detector_seconds * 1e9 / slice_ns)))
    burst = rate_factor == "burst"
    saturate = rate_factor == "sat" or burst
    mean_gap = 0.0 if saturate else slice_ns * 1e-9 / float(rate_factor)
    events = []
    for i in range(len(dets)):
        t = 0.0
        for k in range(n_per):
            t += rng.exponential(mean_gap) if mean_gap > 0 else 0.0
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
    _lib.trig_engine_trace(len(events) + 16)
    deferred = 0
    released_early = False
    if burst:
        # everything staged while the engine holds; a full staging area
        # releases the hold (the engine then drains while the rest arrive)
        _lib.trig_engine_hold(True)
        try:
            for (t, i, k) in events:
                t0, st, cont = pools[i][k % len(pools[i])]
                if not released_early:
                    try:
                        _lib.trig_submit_slice(dets[i], t0, st.hits, st.pmt_off, is_continuation=cont)
                        continue
                    except _lib.TrigError as e:
                        if e.code != _lib.TRIG_EAGAIN:
                            raise
                        released_early = True
                        _lib.trig_engine_hold(False)
                deferred += _submit(dets[i], t0, st, cont)
        finally:
            t_start = time.perf_counter()
            _lib.trig_engine_hold(False)
        for i in range(len(dets)):
            arrivals[i] = [t_start] * n_per
    else:
        # one submitting thread per detector, as each tower's data
        # acquisition feeds the trigger on its own: a large detector's copy
        # does not hold back the others' submissions
        t_start = time.perf_counter()
        deferred_of = [0] * len(dets)

        def submitter(i):
            try:
                for (t, _, k) in (e for e in events if e[1] == i):
                    now = time.perf_counter() - t_start
                    if t > now:
                        time.sleep(t - now)
                    t0, st, cont = pools[i][k % len(pools[i])]
                    arrivals[i][k] = t_start + t
                    deferred_of[i] += _submit(dets[i], t0, st, cont)
            except Exception as err:        # noqa: BLE001
                errors.append(f"detector {i}: submit failed: {err!r}")

        subs = [threading.Thread(target=submitter, args=(i,), daemon=True) for i in range(len(dets))]
        for th in subs:
            th.start()
        for th in subs:
            th.join()
        deferred = sum(deferred_of)
    for th in threads:
        th.join()
    t_end = time.perf_counter()
    trace = _lib.trig_engine_trace_read(len(events) + 16)
    if trace_out:
        np.save(trace_out, trace)           # the engine's per-slice records of this run
    _lib.trig_engine_trace(0)
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
                        "p999_ms": _pct(le, 99.9), "max_ms": max(le) if le else float("nan"), "slices": len(le)})
    wall = t_end - t_start
    return {
        "rate_factor": rate_factor,
        "mode": mode,
        "detector_seconds": detector_seconds,
        "slices": int(sum(len(x) for x in results.values())),
        "bad_status": int(bad),
        "errors": errors,
        "wall_s": wall,
        "hits_per_s": hits / wall if wall > 0 else 0.0,
        "detector_s_per_wall_s": len(dets) * detector_seconds / wall if wall > 0 else 0.0,
        "p50_ms": _pct(lat_e2e, 50),
        "p99_ms": _pct(lat_e2e, 99),
        "p999_ms": _pct(lat_e2e, 99.9),
        "max_ms": max(lat_e2e) if lat_e2e else float("nan"),
        "engine_p99_ms": _pct(lat_engine, 99),
        "budget_ms": slice_ns * 1e-6,
        "deferred_submits": deferred,
        "released_early": released_early if burst else None,
        "per_detector": per_det,
        "trace": trace_summary(trace),
    }


def trace_summary(tr: np.ndarray) -> dict:
    """Where a slice's time goes, from the engine's records: submit (the
    host-to-device copy, and the resident tail's update; copy_wait the part
    spent waiting for the copies after the host work), queue (waiting for
    a slot and a batch), device (the batch's kernels, CUDA events), readback
    (the results' copy back after the counters) -- percentiles of each, and
    the same parts for the slowest 0.1 % of slices."""
    if len(tr) == 0:
        return {}
    ms = 1e-6
    parts = {
        "submit_ms": (tr["t_queued_ns"] - tr["t_submit_ns"]) * ms,
        "copy_wait_ms": tr["copy_wait_us"] * 1e-3,
        "queue_ms": (tr["t_launch_ns"] - tr["t_queued_ns"]) * ms,
        "batch_ms": (tr["t_stats_ns"] - tr["t_launch_ns"]) * ms,
        "readback_ms": (tr["t_done_ns"] - tr["t_stats_ns"]) * ms,
        "total_ms": (tr["t_done_ns"] - tr["t_submit_ns"]) * ms,
    }
    dev = tr["device_ms"][tr["device_ms"] >= 0]
    out = {name: {"p50": _pct(v, 50), "p99": _pct(v, 99), "p999": _pct(v, 99.9)} for name, v in parts.items()}
    out["device_ms"] = {"p50": _pct(dev, 50), "p99": _pct(dev, 99), "p999": _pct(dev, 99.9)}
    out["batch_slices"] = {"mean": float(np.mean(tr["batch_slices"])), "max": int(np.max(tr["batch_slices"]))}
    out["batches"] = int(len(np.unique(tr["batch"])))
    out["continuation_share"] = float(np.mean(tr["continuation"]))
    tot = parts["total_ms"]
    cut = np.percentile(tot, 99.9)
    slow = tot >= cut
    out["slowest"] = {name: float(np.mean(v[slow])) for name, v in parts.items()}
    out["slowest"]["n_pmt"] = sorted(set(int(x) for x in tr["n_pmt"][slow]))
    out["slowest"]["batch_slices"] = float(np.mean(tr["batch_slices"][slow]))
    return out


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else float("nan")


def make_pools(detectors, rates, pool: int, par: dict, seed: int = 0):
    """Per detector: one contiguous run of `pool` slices (with muons), cut
    into the pool's submissions in page-locked memory -- the first with
    both halos, the others from t0 on (continuations)."""
    import workload
    S = par["slice_ns"]
    H = workload.HALO_NS
    pools = []
    for i, (det, rate) in enumerate(zip(detectors, rates)):
        t_origin = workload.T_ORIGIN_NS
        full = workload.gen_stream(det, t_origin - H, t_origin + pool * S + H, rate, n_muons=10 * pool, seed=seed,
                                   stream=5000 + i)
        subs = []
        for k in range(pool):
            t0 = t_origin + k * S
            st = workload.cut(full, t0 - H if k == 0 else t0, t0 + S + H)
            subs.append((t0, workload.Stream(_lib.pinned_copy(st.hits), _lib.pinned_copy(st.pmt_off)), int(k > 0)))
        del full
        pools.append(subs)
    return pools


def _parse_run(text: str):
    rate, mode, secs = text.split(":")
    return (rate if rate in ("sat", "burst") else float(rate)), int(mode), float(secs)


def main():
    import workload

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--runs", nargs="+", default=["4:1:60", "4:0:60", "1:1:30", "sat:1:20", "sat:0:20"],
                    help="rate:mode:detector_seconds per run (rate in units of real time, sat or burst)")
    ap.add_argument("--pool", type=int, default=20, help="contiguous pre-generated slices per detector")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--trace-dir", default=None, help="save each run's per-slice engine trace here (run<k>.npy)")
    ap.add_argument("--detectors", type=int, nargs="+", default=[0, 1, 2, 3],
                    help="which of the four detectors (32, 84, 84, 2688 PMTs) take part")
    args = ap.parse_args()
    par = dict(workload.DEFAULT_PARAMS)
    spec = [(workload.nemo_tower(), 50e3), (workload.km3_tower(), 55e3), (workload.km3_tower(), 55e3),
            (workload.tower_array(), 55e3)]
    spec = [spec[i] for i in args.detectors]
    t = time.perf_counter()
    pools = make_pools([d for d, _ in spec], [r for _, r in spec], args.pool, par, args.seed)
    gen_s = time.perf_counter() - t
    dets = [_lib.Detector(d.xyz_mm, d.floor_id, par) for d, _ in spec]
    runs = []
    for k, text in enumerate(args.runs):
        rate, mode, secs = _parse_run(text)
        out_k = None
        if args.trace_dir:
            os.makedirs(args.trace_dir, exist_ok=True)
            out_k = os.path.join(args.trace_dir, f"run{k}.npy")
        runs.append(replay(dets, pools, rate, secs, par["slice_ns"], args.seed + k, mode, trace_out=out_k))
        print(json.dumps(runs[-1]), file=sys.stderr, flush=True)      # progress, one line per run
    out = {"detectors": ", ".join(f"{d.n_pmt}@{r / 1e3:g}kHz" for d, r in spec), "pool_slices_per_detector": args.pool,
           "pool_generation_s": gen_s, "continuation": "every pool slice after the first", "runs": runs}
    for d in dets:
        d.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
