"""trig_batch_run_noalloc: the batch path for callers that cannot allocate
device memory (a trigger node's real-time thread, code running beside a
global-mode CUDA graph capture).  Its scratch is the library's static
device array; its results must equal trig_batch_run's, call after call.

Kept in a file of its own that runs after the other GPU tests; it passes
alone in a fresh process and after them.
"""
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


def test_noalloc_matches_batch_run_twice(pkg, params):
    import torch
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn

    nemo = workload.cfg_nemo()
    km3 = workload.cfg_km3()
    dets = [pkg.Detector(w.detectors[0].xyz_mm, w.detectors[0].floor_id, params) for w in (nemo, km3)]
    slices = [SliceIn(dets[0], s.t0, s.stream.hits, s.stream.pmt_off) for s in nemo.submissions]
    slices += [SliceIn(dets[1], s.t0, s.stream.hits, s.stream.pmt_off) for s in km3.submissions[:2]]

    ref = DeviceBatch(slices)
    ref.run()
    want = _outputs(ref)
    assert all(o[0]["status"] == 0 for o in want)
    assert sum(len(o[1]) for o in want) > 0

    # the no-allocation path writes into a second set of outputs
    out = DeviceBatch(slices)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        for t in out.trig + out.win + [out.stats]:
            t.fill_(0xA5)                      # stale bytes must not leak into results
        _lib.trig_batch_run_noalloc(out.descs, stream)
        got = _outputs(out)
        for k, (g, w) in enumerate(zip(got, want)):
            assert g[0] == w[0], (call, k)
            assert np.array_equal(g[1], w[1]), (call, k)
            assert np.array_equal(g[2], w[2]), (call, k)
    for d in dets:
        d.close()


def test_noalloc_rejects_a_batch_beyond_the_static_scratch(pkg, params):
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn

    g = workload.nemo_tower()
    det = pkg.Detector(g.xyz_mm, g.floor_id, params)
    t0 = workload.T_ORIGIN_NS
    # ~5 M hits: its staging alone exceeds the 64 MiB array
    st = workload.gen_stream(g, t0 - 3000, t0 + params["slice_ns"] + 3000, 800e3, seed=2)
    batch = DeviceBatch([SliceIn(det, t0, st.hits, st.pmt_off)])
    with pytest.raises(_lib.TrigError) as e:
        _lib.trig_batch_run_noalloc(batch.descs)
    assert e.value.code == _lib.TRIG_ECAPACITY
    with pytest.raises(_lib.TrigError) as e:
        _lib.trig_batch_run_noalloc(batch.descs * (_lib.NOALLOC_MAX_SLICES + 1))
    assert e.value.code == _lib.TRIG_EINVAL
    det.close()
