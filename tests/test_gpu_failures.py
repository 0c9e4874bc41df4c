"""Failure paths of the engine and the tile pass, made on the host or by a
device wait that runs out; nothing faults, traps or hangs the GPU.

* admission full: a staging limit set through the C ABI makes a submission
  return TRIG_EAGAIN, and the slice goes through once memory frees up;
* allocation failure: the result pool's next request fails (host-side
  injection), the slice completes with TRIG_ENOMEM and no arrays, the next
  one is exact;
* bounded device wait: with the stagers told to stage nothing, the tile
  pass's first wait runs out after a short limit (no copy in flight), the
  slices report TRIG_ETIMEOUT with no output, and the same slices run
  exactly afterwards.
"""
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


@pytest.fixture(scope="module")
def km3(params):
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0], threads=0)
    return wl, ref


def _same(r, ref, ctx):
    assert r.status == 0, (ctx, r.status, r.flags)
    assert r.n_seeds == len(ref.seeds), ctx
    for f in ("t", "pmt", "charge", "count"):
        assert np.array_equal(r.triggers[f], ref.triggers[f]), (ctx, f)
    for f in ("lo", "hi", "n_hits", "n_triggers"):
        assert np.array_equal(r.windows[f], ref.windows[f]), (ctx, f)


def test_submit_returns_eagain_when_staging_is_full(pkg, params, km3):
    wl, ref = km3
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    s0, s1 = wl.submissions[0], wl.submissions[1]
    one = int(s0.stream.hits.nbytes + s0.stream.pmt_off.nbytes)
    pkg.trig_engine_set_mode(1)
    pkg.trig_engine_hold(True)
    try:
        # room for one slice's staging block (a power-of-two class) only
        cls = 1 << 16
        while cls < one:
            cls <<= 1
        pkg.trig_engine_set_staging_limit(cls + cls // 2)
        pkg.trig_submit_slice(det, s0.t0, s0.stream.hits, s0.stream.pmt_off)
        with pytest.raises(pkg.TrigError) as e:
            pkg.trig_submit_slice(det, s1.t0, s1.stream.hits, s1.stream.pmt_off)
        assert e.value.code == pkg.TRIG_EAGAIN
    finally:
        pkg.trig_engine_hold(False)
    _same(pkg.trig_poll(det, 60_000), ref[0], "first slice")
    # its block is back: the second submission fits now
    pkg.trig_submit_slice(det, s1.t0, s1.stream.hits, s1.stream.pmt_off)
    pkg.trig_engine_set_staging_limit(0)
    _same(pkg.trig_poll(det, 60_000), ref[1], "second slice after the retry")
    det.close()


def test_result_allocation_failure_gives_enomem(pkg, params, km3):
    wl, ref = km3
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    pkg.trig_engine_set_mode(1)
    s0, s1 = wl.submissions[0], wl.submissions[1]
    pkg.trig_engine_fail_result_allocs(1)
    try:
        pkg.trig_submit_slice(det, s0.t0, s0.stream.hits, s0.stream.pmt_off)
        r = pkg.trig_poll(det, 60_000)
    finally:
        pkg.trig_engine_fail_result_allocs(0)
    assert r.status == pkg.TRIG_ENOMEM
    assert len(r.triggers) == 0 and len(r.windows) == 0
    pkg.trig_submit_slice(det, s1.t0, s1.stream.hits, s1.stream.pmt_off)
    _same(pkg.trig_poll(det, 60_000), ref[1], "slice after the failure")
    det.close()


def test_device_wait_runs_out_and_the_device_stays_usable(pkg, params, km3):
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    wl, ref = km3
    g = wl.detectors[0]
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    subs = wl.submissions[:2]
    batch = DeviceBatch([SliceIn(det, s.t0, s.stream.hits, s.stream.pmt_off) for s in subs])
    pkg.trig_set_device_wait(2_000_000, stall=True)           # 2 ms, nothing staged
    try:
        batch.run()
        res = batch.results()
        # the engine's batches take the same path
        pkg.trig_engine_set_mode(1)
        pkg.trig_submit_slice(det, subs[0].t0, subs[0].stream.hits, subs[0].stream.pmt_off)
        r_engine = pkg.trig_poll(det, 60_000)
    finally:
        pkg.trig_set_device_wait(0, stall=False)
    for stats, trig, win in res:
        assert int(stats["status"]) == pkg.TRIG_ETIMEOUT
        assert int(stats["flags"]) & pkg.TRIG_FLAG_TIMEOUT
        assert int(stats["n_triggers"]) == 0 and int(stats["n_windows"]) == 0
        assert len(trig) == 0 and len(win) == 0
    assert r_engine.status == pkg.TRIG_ETIMEOUT and len(r_engine.triggers) == 0
    # the same slices, run again, are exact
    batch.run()
    for k, (stats, trig, win) in enumerate(batch.results()):
        assert int(stats["status"]) == 0
        assert np.array_equal(trig["t"], ref[k].triggers["t"])
        assert np.array_equal(trig["count"], ref[k].triggers["count"])
        assert np.array_equal(win["n_hits"], ref[k].windows["n_hits"])
    det.close()


def test_device_wait_parameters_checked(pkg):
    lib = pkg.load()
    try:
        assert lib.trig_set_device_wait(0, 2) == pkg.TRIG_EINVAL
        assert lib.trig_set_device_wait(0, -1) == pkg.TRIG_EINVAL
        assert lib.trig_set_device_wait(601 * 10**9, 0) == pkg.TRIG_EINVAL
        assert lib.trig_engine_hold(2) == pkg.TRIG_EINVAL
    finally:
        pkg.trig_set_device_wait(0, stall=False)
        pkg.trig_engine_hold(False)
