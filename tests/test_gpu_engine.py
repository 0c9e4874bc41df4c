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
    """Four detectors (32, 84, 84, 2688 PMTs) submitted interleaved while the
    engine holds admission, so that they share one batch: each result
    equals the same slice run alone (tolerance 0), and every detector's
    results equal the oracle."""
    wl = workload.cfg_serving_pool(slices_per_det=2)
    dets = [pkg.Detector(g.xyz_mm, g.floor_id, params) for g in wl.detectors]
    pkg.trig_engine_set_mode(1)
    # alone: one slice at a time, waiting for each result
    alone = {}
    for i, s in enumerate(wl.submissions):
        pkg.trig_submit_slice(dets[s.det_index], s.t0, s.stream.hits, s.stream.pmt_off)
        alone[i] = pkg.trig_poll(dets[s.det_index], 60_000)
    # mixed: everything interleaved, admitted at once
    rng = np.random.Generator(np.random.PCG64(4))
    by_det = {}
    for i in range(len(wl.submissions)):
        by_det.setdefault(wl.submissions[i].det_index, []).append(i)
    seq = []
    while any(by_det.values()):
        d = int(rng.choice([k for k, v in by_det.items() if v]))
        seq.append(by_det[d].pop(0))
    b0, s0 = pkg.trig_engine_stats()
    pkg.trig_engine_hold(True)
    try:
        for i in seq:
            s = wl.submissions[i]
            pkg.trig_submit_slice(dets[s.det_index], s.t0, s.stream.hits, s.stream.pmt_off)
    finally:
        pkg.trig_engine_hold(False)
    mixed = {}
    for d_index, det in enumerate(dets):
        for i in [j for j in range(len(wl.submissions)) if wl.submissions[j].det_index == d_index]:
            mixed[i] = pkg.trig_poll(det, 120_000)
    b1, s1 = pkg.trig_engine_stats()
    assert s1 - s0 == len(seq)
    assert b1 - b0 == 1, (b1 - b0, s1 - s0)           # one batch held every detector's slices
    for i in alone:
        a, m = alone[i], mixed[i]
        assert a.status == 0 and m.status == 0
        assert a.n_seeds == m.n_seeds
        assert np.array_equal(a.triggers, m.triggers)
        assert np.array_equal(a.windows, m.windows)
    # every detector against the oracle
    for k, g in enumerate(wl.detectors):
        ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[k].hits, wl.run_slices[k], threads=0)
        idx = [j for j in range(len(wl.submissions)) if wl.submissions[j].det_index == k]
        assert len(idx) == len(ref) == 2
        for r_i, j in enumerate(idx):
            _same(mixed[j], ref[r_i], f"det {k} ({g.n_pmt} PMTs) slice {r_i}")
    for d in dets:
        d.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_engine_continuation_matches_oracle(pkg, params, mode):
    """Contiguous slices of two detectors, interleaved: the first slice of
    each run carries both halos, the later ones start at t0 and ask the
    library for the leading halo it kept on the device
    (is_continuation = 1).  Every result equals the oracle on the whole
    run."""
    pkg.trig_engine_set_mode(mode)
    wl = workload.cfg_serving_pool(slices_per_det=4, dets=[("nemo", 120e3), ("km3", 55e3)])
    dets = [pkg.Detector(g.xyz_mm, g.floor_id, params) for g in wl.detectors]
    halo = dets[0].halo_ns
    S = params["slice_ns"]
    order = []
    for k in range(4):
        for d in (0, 1):
            order.append((d, k))
    for d, k in order:
        t0 = wl.run_slices[d][k]
        if k == 0:
            st = workload.cut(wl.runs[d], t0 - halo, t0 + S + halo)
            pkg.trig_submit_slice(dets[d], t0, st.hits, st.pmt_off)
        else:
            st = workload.cut(wl.runs[d], t0, t0 + S + halo)
            pkg.trig_submit_slice(dets[d], t0, st.hits, st.pmt_off, is_continuation=1)
    for d, g in enumerate(wl.detectors):
        ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[d].hits, wl.run_slices[d], threads=0)
        for k in range(4):
            r = pkg.trig_poll(dets[d], 60_000)
            assert r is not None
            _same(r, ref[k], f"mode {mode} det {d} slice {k}")
            want_hits = int(np.count_nonzero((wl.runs[d].hits["t"] >= wl.run_slices[d][k] - halo) &
                                             (wl.runs[d].hits["t"] < wl.run_slices[d][k] + S + halo)))
            assert r.n_hits == want_hits
    for det in dets:
        det.close()
    pkg.trig_engine_set_mode(1)


def test_engine_continuation_refused(pkg, params):
    """A continuation needs a previous submission of the detector, the next
    t0, and no hit before t0; each case is refused (EINVAL) and leaves the
    resident tail usable."""
    wl = workload.cfg_serving_pool(slices_per_det=3, dets=[("nemo", 80e3)])
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    halo, S = det.halo_ns, params["slice_ns"]
    t0s = wl.run_slices[0]
    full = wl.runs[0]
    st1 = workload.cut(full, t0s[1], t0s[1] + S + halo)
    with pytest.raises(pkg.TrigError) as e:                  # nothing submitted yet
        pkg.trig_submit_slice(det, t0s[1], st1.hits, st1.pmt_off, is_continuation=1)
    assert e.value.code == pkg.TRIG_EINVAL
    st0 = workload.cut(full, t0s[0] - halo, t0s[0] + S + halo)
    pkg.trig_submit_slice(det, t0s[0], st0.hits, st0.pmt_off)
    st2 = workload.cut(full, t0s[2], t0s[2] + S + halo)
    with pytest.raises(pkg.TrigError) as e:                  # not the next slice
        pkg.trig_submit_slice(det, t0s[2], st2.hits, st2.pmt_off, is_continuation=1)
    assert e.value.code == pkg.TRIG_EINVAL
    with_halo = workload.cut(full, t0s[1] - halo, t0s[1] + S + halo)
    with pytest.raises(pkg.TrigError) as e:                  # carries its own leading halo
        pkg.trig_submit_slice(det, t0s[1], with_halo.hits, with_halo.pmt_off, is_continuation=1)
    assert e.value.code == pkg.TRIG_EINVAL
    pkg.trig_submit_slice(det, t0s[1], st1.hits, st1.pmt_off, is_continuation=1)
    ref = oracle.run(g.xyz_mm, g.floor_id, params, full.hits, t0s[:2])
    for k in range(2):
        _same(pkg.trig_poll(det, 60_000), ref[k], f"slice {k}")
    det.close()


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
