"""trig_batch_run_noalloc: the batch path for callers that cannot allocate
device memory (a trigger node's real-time thread, code running beside a
global-mode CUDA graph capture).  Its scratch is the library's static
device array; its results must equal trig_batch_run's, call after call,
whatever the previous call left in the array.

Kept in a file of its own that runs after the other GPU tests; it passes
alone in a fresh process and after them.
"""
import threading

import numpy as np
import pytest

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


def _outputs(batch):
    res = batch.results()
    return [(dict(zip(s.dtype.names, (int(s[f]) for f in s.dtype.names))), t.copy(), w.copy()) for s, t, w in res]


def _batches(pkg, params):
    """Two different batches: NEMO plus two KM3Net-It slices, and a wide
    detector (168 PMTs, bucketed staging) with a KM3Net-It slice."""
    from paper_1411_3968_gb300.runner import SliceIn
    nemo, km3 = workload.cfg_nemo(), workload.cfg_km3()
    dets = [pkg.Detector(w.detectors[0].xyz_mm, w.detectors[0].floor_id, params) for w in (nemo, km3)]
    a = [SliceIn(dets[0], s.t0, s.stream.hits, s.stream.pmt_off) for s in nemo.submissions]
    a += [SliceIn(dets[1], s.t0, s.stream.hits, s.stream.pmt_off) for s in km3.submissions[:2]]
    wide = workload.tower_array(nx=2, ny=1)
    par_w = dict(params, slice_ns=2_000_000)
    dw = pkg.Detector(wide.xyz_mm, wide.floor_id, par_w)
    t0 = workload.T_ORIGIN_NS
    st = workload.gen_stream(wide, t0 - 3000, t0 + par_w["slice_ns"] + 3000, 200e3, n_muons=20, seed=7)
    b = [SliceIn(dw, t0, st.hits, st.pmt_off)]
    b += [SliceIn(dets[1], s.t0, s.stream.hits, s.stream.pmt_off) for s in km3.submissions[3:4]]
    return dets + [dw], a, b


def test_noalloc_matches_batch_run_across_calls(pkg, params):
    import torch
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch

    dets, a, b = _batches(pkg, params)
    want = {}
    for name, sl in (("a", a), ("b", b)):
        ref = DeviceBatch(sl)
        ref.run()
        want[name] = _outputs(ref)
        assert all(o[0]["status"] == 0 for o in want[name]), name
        assert sum(len(o[1]) for o in want[name]) > 0, name
    # the no-allocation path writes into second sets of outputs; batch b
    # runs between the two calls of batch a, so that a's second call starts
    # from b's leftovers in the static array
    out = {"a": DeviceBatch(a), "b": DeviceBatch(b)}
    stream = torch.cuda.Stream()
    for call, name in enumerate(("a", "b", "a", "b")):
        o = out[name]
        for t in o.trig + o.win + [o.stats]:
            t.fill_(0xA5)                      # stale bytes must not leak into results
        torch.cuda.synchronize()
        _lib.trig_batch_run_noalloc(o.descs, stream.cuda_stream)
        stream.synchronize()
        got = _outputs(o)
        for k, (g, w) in enumerate(zip(got, want[name])):
            assert g[0] == w[0], (call, name, k)
            assert np.array_equal(g[1], w[1]), (call, name, k)
            assert np.array_equal(g[2], w[2]), (call, name, k)
    for d in dets:
        d.close()


def test_noalloc_rejects_a_batch_beyond_the_static_scratch(pkg, params):
    import torch
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn

    g = workload.nemo_tower()
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    t0 = workload.T_ORIGIN_NS
    # ~5 M hits: its staging alone exceeds the 64 MiB array
    st = workload.gen_stream(g, t0 - 3000, t0 + params["slice_ns"] + 3000, 800e3, seed=2)
    batch = DeviceBatch([SliceIn(det, t0, st.hits, st.pmt_off)])
    stream = torch.cuda.Stream()
    with pytest.raises(_lib.TrigError) as e:
        _lib.trig_batch_run_noalloc(batch.descs, stream.cuda_stream)
    assert e.value.code == _lib.TRIG_ECAPACITY
    with pytest.raises(_lib.TrigError) as e:
        _lib.trig_batch_run_noalloc(batch.descs * (_lib.NOALLOC_MAX_SLICES + 1), stream.cuda_stream)
    assert e.value.code == _lib.TRIG_EINVAL
    det.close()


def test_noalloc_refuses_the_legacy_stream_and_capture(pkg, params):
    """The legacy default stream is refused, and so is a stream that is
    capturing a graph (relaxed mode here): nothing is launched, and the
    capture ends normally and is discarded without a replay."""
    import torch
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn

    nemo = workload.cfg_nemo()
    det = pkg.Detector(nemo.detectors[0].xyz_mm, nemo.detectors[0].floor_id, params)
    batch = DeviceBatch([SliceIn(det, s.t0, s.stream.hits, s.stream.pmt_off) for s in nemo.submissions])
    torch.cuda.synchronize()
    with pytest.raises(_lib.TrigError) as e:
        _lib.trig_batch_run_noalloc(batch.descs, 0)
    assert e.value.code == _lib.TRIG_EINVAL
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    refused = []
    with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
        try:
            _lib.trig_batch_run_noalloc(batch.descs, side.cuda_stream)
        except _lib.TrigError as err:
            refused.append(err.code)
    assert refused == [_lib.TRIG_EINVAL]
    del graph
    det.close()


def test_noalloc_beside_another_threads_global_capture(pkg, params):
    """One thread holds a global-mode capture on its own stream while
    another runs the no-allocation call on a non-blocking stream: both
    succeed, and the results equal trig_batch_run's."""
    import torch
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn

    km3 = workload.cfg_km3()
    det = pkg.Detector(km3.detectors[0].xyz_mm, km3.detectors[0].floor_id, params)
    sl = [SliceIn(det, s.t0, s.stream.hits, s.stream.pmt_off) for s in km3.submissions[:2]]
    ref = DeviceBatch(sl)
    ref.run()
    want = _outputs(ref)
    out = DeviceBatch(sl)
    run_stream = torch.cuda.Stream()
    _lib.trig_batch_run_noalloc(out.descs, run_stream.cuda_stream)     # first call: set-up, before any capture
    run_stream.synchronize()
    x = torch.zeros(1024, device="cuda")
    cap_stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    started, done = threading.Event(), threading.Event()
    errors = []

    def capturer():
        try:
            with torch.cuda.graph(graph, stream=cap_stream, capture_error_mode="global"):
                x.add_(1.0)
                started.set()
                done.wait(60)
                x.mul_(2.0)
        except Exception as err:            # noqa: BLE001
            errors.append(("capture", repr(err)))
            started.set()

    th = threading.Thread(target=capturer)
    th.start()
    started.wait(60)
    try:
        _lib.trig_batch_run_noalloc(out.descs, run_stream.cuda_stream)
    except Exception as err:                # noqa: BLE001
        errors.append(("noalloc", repr(err)))
    done.set()
    th.join(120)
    assert not errors, errors
    run_stream.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 2.0
    got = _outputs(out)
    for k, (g, w) in enumerate(zip(got, want)):
        assert g[0] == w[0], k
        assert np.array_equal(g[1], w[1]) and np.array_equal(g[2], w[2]), k
    det.close()
