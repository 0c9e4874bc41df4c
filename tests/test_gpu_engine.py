"""The host-buffer engine (trig_submit_slice / trig_poll) against the oracle:
plain and batched modes, several detectors interleaved (continuous
batching), and each slice's result alone versus in the mix."""
import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    import paper_1411_3968_gb300 as p
    from paper_1411_3968_gb300 import build
    build.build()
    p.load()
    torch.cuda.init()
    return p


def _same(r, ref, ctx):
    assert r.status == 0, (ctx, r.status, r.flags)
    assert r.n_seeds == len(ref.seeds), ctx
    for f in ("t", "pmt", "charge", "count"):
        assert np.array_equal(r.triggers[f], ref.triggers[f]), (ctx, f)
    for f in ("lo", "hi", "n_hits", "n_triggers"):
        assert np.array_equal(r.windows[f], ref.windows[f]), (ctx, f)


@pytest.mark.parametrize("mode", [0, 1])
def test_engine_km3_matches_oracle(pkg, params, mode):
    pkg.trig_engine_set_mode(mode)
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    ids = [pkg.trig_submit_slice(det, s.t0, s.stream.hits, s.stream.pmt_off) for s in wl.submissions]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    for k, sid in enumerate(ids):
        r = pkg.trig_poll(det, 60_000)
        assert r is not None and r.slice_id == sid
        _same(r, ref[k], f"mode {mode} slice {k}")
        assert r.latency_ns > 0
    assert pkg.trig_poll(det, 0) is None
    det.close()
    pkg.trig_engine_set_mode(1)


def test_engine_from_page_locked_buffers(pkg, params):
    """Slices submitted from trig_host_alloc memory (pinned_copy) give the
    oracle's results; the buffers may be overwritten once submit returns."""
    pkg.trig_engine_set_mode(1)
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    bufs = [(pkg.pinned_copy(s.stream.hits), pkg.pinned_copy(s.stream.pmt_off)) for s in wl.submissions]
    assert all(np.array_equal(h, s.stream.hits) for (h, _), s in zip(bufs, wl.submissions))
    for (h, o), s in zip(bufs, wl.submissions):
        pkg.trig_submit_slice(det, s.t0, h, o)
        h["t"] = 0                                   # the copy was taken before submit returned
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    for k in range(len(ref)):
        r = pkg.trig_poll(det, 60_000)
        assert r is not None
        _same(r, ref[k], f"pinned slice {k}")
    det.close()


def test_engine_alone_equals_in_mix(pkg, params):
    """Four detectors (32, 84, 84, 2688 PMTs) submitted interleaved share
    batches; each result equals the same slice run alone (tolerance 0)."""
    wl = workload.cfg_serving_pool(slices_per_det=2)
    dets = [pkg.Detector(g.xyz_mm, g.floor_id, params) for g in wl.detectors]
    pkg.trig_engine_set_mode(1)
    # alone: one slice at a time, waiting for each result
    alone = {}
    for i, s in enumerate(wl.submissions):
        pkg.trig_submit_slice(dets[s.det_index], s.t0, s.stream.hits, s.stream.pmt_off)
        alone[i] = pkg.trig_poll(dets[s.det_index], 60_000)
    # mixed: everything at once
    order = list(range(len(wl.submissions)))
    rng = np.random.Generator(np.random.PCG64(4))
    by_det = {}
    for i in order:
        by_det.setdefault(wl.submissions[i].det_index, []).append(i)
    seq = []
    while any(by_det.values()):
        d = int(rng.choice([k for k, v in by_det.items() if v]))
        seq.append(by_det[d].pop(0))
    for i in seq:
        s = wl.submissions[i]
        pkg.trig_submit_slice(dets[s.det_index], s.t0, s.stream.hits, s.stream.pmt_off)
    mixed = {}
    for i in seq:
        pass
    for d_index, det in enumerate(dets):
        for i in [j for j in range(len(wl.submissions)) if wl.submissions[j].det_index == d_index]:
            mixed[i] = pkg.trig_poll(det, 120_000)
    for i in alone:
        a, m = alone[i], mixed[i]
        assert a.status == 0 and m.status == 0
        assert a.n_seeds == m.n_seeds
        assert np.array_equal(a.triggers, m.triggers)
        assert np.array_equal(a.windows, m.windows)
    # and one detector against the oracle
    k = 1
    g = wl.detectors[k]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[k].hits, wl.run_slices[k])
    idx = [j for j in range(len(wl.submissions)) if wl.submissions[j].det_index == k]
    for r_i, j in enumerate(idx):
        _same(mixed[j], ref[r_i], f"det {k} slice {r_i}")
    for d in dets:
        d.close()


def test_engine_rejects_bad_offsets(pkg, params):
    g = workload.nemo_tower()
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    off = np.zeros(33, np.uint64)
    off[5] = 3
    with pytest.raises(pkg.TrigError):
        pkg.trig_submit_slice(det, 0, np.zeros(3, workload.HIT_DTYPE), off)   # decreasing offsets
    det.close()


def test_graph_replay_after_a_smaller_launch_of_the_same_kernel(pkg, params):
    """A graph captured for a batch that needs more shared memory is
    replayed after a smaller launch of the same tile kernel; the kernel's
    shared-memory limit must still admit the graph's launch."""
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    km3, nemo = workload.cfg_km3(), workload.cfg_nemo()
    dk = pkg.Detector(km3.detectors[0].xyz_mm, km3.detectors[0].floor_id, params)
    dn = pkg.Detector(nemo.detectors[0].xyz_mm, nemo.detectors[0].floor_id, params)
    big = DeviceBatch([SliceIn(dk, s.t0, s.stream.hits, s.stream.pmt_off) for s in km3.submissions[:1]])
    small = DeviceBatch([SliceIn(dn, s.t0, s.stream.hits, s.stream.pmt_off) for s in nemo.submissions])
    big.run(graph=True)
    first = big.results()
    small.run()
    small.results()
    big.run(graph=True)
    again = big.results()
    ref = oracle.run(km3.detectors[0].xyz_mm, km3.detectors[0].floor_id, params, km3.runs[0].hits,
                     km3.run_slices[0][:1])[0]
    for res in (first, again):
        stats, trig, win = res[0]
        assert int(stats["status"]) == 0
        assert np.array_equal(trig["t"], ref.triggers["t"]) and np.array_equal(win["n_hits"], ref.windows["n_hits"])
    dk.close()
    dn.close()


def test_engine_event_payload(pkg, params):
    """trig_set_events: engine results carry the hits inside their windows."""
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    pkg.trig_set_events(det, True)
    pkg.trig_engine_set_mode(1)
    for s in wl.submissions:
        pkg.trig_submit_slice(det, s.t0, s.stream.hits, s.stream.pmt_off)
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    for k in range(len(ref)):
        r = pkg.trig_poll(det, 60_000)
        _same(r, ref[k], f"slice {k}")
        want = oracle.events(wl.runs[0].hits, ref[k].windows)
        assert r.n_events == len(want) == len(r.events)
        for f in ("t", "pmt", "charge"):
            assert np.array_equal(r.events[f], want[f]), (k, f)
    det.close()


@pytest.mark.parametrize("extra", [dict(l0_hits=7, l0_window_ns=1000), dict(seed_rule=1, threshold=1),
                                   dict(count_distinct_pmts=1)], ids=["level0", "ladder", "distinct"])
def test_engine_with_the_paper_rules(pkg, params, extra):
    """The engine's batches take the extended-rule tile kernel when a
    detector uses level 0, the coincidence ladder or the distinct count:
    results equal the oracle."""
    pkg.trig_engine_set_mode(1)
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    par = dict(params, **extra)
    det = pkg.Detector(g.xyz_mm, g.floor_id, par, tower_id=g.tower_id)
    for s in wl.submissions:
        pkg.trig_submit_slice(det, s.t0, s.stream.hits, s.stream.pmt_off)
    ref = oracle.run(g.xyz_mm, g.floor_id, par, wl.runs[0].hits, wl.run_slices[0], tower_id=g.tower_id)
    for k in range(len(ref)):
        r = pkg.trig_poll(det, 60_000)
        assert r is not None
        _same(r, ref[k], f"{extra} slice {k}")
    det.close()
