"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Timestamps and dt_max are integer ns, so trigger lists, counts and windows
must match bit-exactly; the merged order and seed counts are compared row by
row.  Inputs are seeded synthetic workloads (workload/) and hand-built
slices at every boundary of the trigger rule.
"""
import glob
import json
import os

import numpy as np
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GEOM = {"nemo32": workload.nemo_tower, "km3it84": workload.km3_tower, "array2688": workload.tower_array}


@pytest.fixture(scope="module")
def pkg():
    import torch
    import paper_1411_3968_gb300 as p
    from paper_1411_3968_gb300 import build
    build.build()
    p.load()
    torch.cuda.init()
    return p


def _det(pkg, geom, par):
    return pkg.Detector(geom.xyz_mm, geom.floor_id, par, tower_id=geom.tower_id)


def _run(pkg, det, subs, graph=False, each=False):
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    b = DeviceBatch([SliceIn(det if not isinstance(det, list) else det[i], t0, s.hits, s.pmt_off)
                     for i, (t0, s) in enumerate(subs)])
    if each:
        b.run_each()
    else:
        b.run(graph=graph)
    return b, b.results()


def _assert_same(res, ref, ctx=""):
    stats, trig, win = res
    assert int(stats["status"]) == 0, (ctx, stats)
    assert int(stats["n_seeds"]) == len(ref.seeds), ctx
    assert len(trig) == len(ref.triggers), (ctx, len(trig), len(ref.triggers))
    for f in ("t", "pmt", "charge", "count"):
        assert np.array_equal(trig[f], ref.triggers[f]), (ctx, f)
    assert len(win) == len(ref.windows), ctx
    for f in ("lo", "hi", "n_hits", "n_triggers"):
        assert np.array_equal(win[f], ref.windows[f]), (ctx, f)


def _subs_from_run(full, t0s, slice_ns, halo=3000):
    return [(t0, workload.cut(full, t0 - halo, t0 + slice_ns + halo)) for t0 in t0s]


def _stream_from_hits(hits, n_pmt):
    h = np.sort(hits, order=["pmt", "t", "charge"], kind="stable")
    off = np.zeros(n_pmt + 1, np.uint64)
    np.cumsum(np.bincount(h["pmt"], minlength=n_pmt), out=off[1:])
    return workload.Stream(h, off)


# --------------------------------------------------------------------- dt_max

@pytest.mark.parametrize("name", ["nemo32", "km3it84", "array2688"])
def test_dtmax_table_bit_exact(pkg, params, name):
    g = GEOM[name]()
    d = _det(pkg, g, params)
    assert np.array_equal(d.dtmax(), oracle.dtmax(g.xyz_mm, params))
    d.close()


def test_dtmax_random_geometry(pkg, params):
    rng = np.random.Generator(np.random.PCG64(12))
    xyz = rng.integers(-2_000_000, 2_000_000, size=(600, 3)).astype(np.int32)
    xyz[100:120] = xyz[0]
    fl = np.arange(600, dtype=np.uint32)
    for par in (params, dict(params, n_num=1, n_den=1, tol_ns=0), dict(params, n_num=9999, n_den=7, tol_ns=3)):
        d = pkg.Detector(xyz, fl, par)
        assert np.array_equal(d.dtmax(), oracle.dtmax(xyz, par))
        d.close()


# --------------------------------------------------------------------- golden

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))), ids=os.path.basename)
def test_golden_fixtures_on_gpu(pkg, params, path):
    fx = json.load(open(path))
    g = GEOM[fx["geometry"]]()
    par = dict(params)
    par.update(fx["params"])
    hits = np.zeros(len(fx["hits"]), workload.HIT_DTYPE)
    for i, (t, p, q) in enumerate(fx["hits"]):
        hits[i] = (t, p, q, 0)
    full = _stream_from_hits(hits, g.n_pmt)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, _subs_from_run(full, fx["slices"], par["slice_ns"]))
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, fx["slices"])
    for r, o, exp in zip(res, ref, fx["expected"]):
        _assert_same(r, o, path)
        assert [tuple(int(x[f]) for f in ("t", "pmt", "charge", "count")) for x in r[1]] == \
            [tuple(x) for x in exp["triggers"]]
    d.close()


# --------------------------------------------------------------- random tiny

@pytest.mark.parametrize("case", range(8))
def test_random_dense_slices(pkg, params, case):
    rng = np.random.Generator(np.random.PCG64(500 + case))
    g = [workload.nemo_tower, workload.km3_tower][case % 2]()
    par = dict(params)
    par["slice_ns"] = int(rng.choice([20_000, 100_000, 1_000_000]))
    par["threshold"] = int(rng.integers(1, 7))
    par["q_seed_adc"] = int(rng.choice([300, 150, 65535]))
    if case >= 6:
        par.update(corr_window_ns=700, win_half_ns=int(rng.integers(0, 2000)), floor_tau_ns=int(rng.integers(0, 60)))
    t0 = 5_000_000
    n = int(rng.integers(200, 4000))
    t = rng.integers(t0 - 3000, t0 + 2 * par["slice_ns"] + 3000, n)
    t[: n // 4] = t[n // 4: 2 * (n // 4)] + rng.integers(-30, 31, n // 4)
    t[-20:] = t[-40:-20]
    hits = np.zeros(n, workload.HIT_DTYPE)
    hits["t"] = t
    hits["pmt"] = rng.integers(0, g.n_pmt, n)
    hits["charge"] = rng.integers(1, 500, n)
    t0s = [t0, t0 + par["slice_ns"]]
    full = _stream_from_hits(hits, g.n_pmt)
    halo = max(par["corr_window_ns"], par["win_half_ns"], par["floor_tau_ns"])
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, _subs_from_run(full, t0s, par["slice_ns"], halo))
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, t0s)
    for k, (r, o) in enumerate(zip(res, ref)):
        _assert_same(r, o, f"case {case} slice {k}")
    d.close()


# ------------------------------------------------------------------ configs

def test_nemo_config(pkg, params):
    wl = workload.cfg_nemo()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    b, res = _run(pkg, d, [(s.t0, s.stream) for s in wl.submissions])
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    _assert_same(res[0], ref[0], "nemo")
    # row level: merged order (k-way merge), seeds and their counts
    merged, seedcnt = b.rows(0)
    own = wl.runs[0].hits
    own = own[(own["t"] >= wl.run_slices[0][0]) & (own["t"] < wl.run_slices[0][0] + params["slice_ns"])]
    om = oracle.merge(own)
    for f in ("t", "pmt", "charge"):
        assert np.array_equal(merged[f], om[f]), f
    is_seed = seedcnt != 0xFFFFFFFF
    assert is_seed.sum() == len(ref[0].seeds)
    assert np.array_equal(merged["t"][is_seed], ref[0].seeds["t"])
    assert np.array_equal(seedcnt[is_seed], ref[0].seeds["count"])
    d.close()


def test_km3_config_five_slices_with_bursts(pkg, params):
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    subs = [(s.t0, s.stream) for s in wl.submissions]
    _, res = _run(pkg, d, subs)
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    for k in range(len(subs)):
        _assert_same(res[k], ref[k], f"km3 slice {k}")
    # plain per-slice launches and the graph replay give the same
    _, res_each = _run(pkg, d, subs, each=True)
    _, res_graph = _run(pkg, d, subs, graph=True)
    for k in range(len(subs)):
        _assert_same(res_each[k], ref[k], f"km3 each {k}")
        _assert_same(res_graph[k], ref[k], f"km3 graph {k}")
    d.close()


def test_scaled_array_config(pkg, params):
    wl = workload.cfg_scaled()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    _, res = _run(pkg, d, [(s.t0, s.stream) for s in wl.submissions])
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    _assert_same(res[0], ref[0], "scaled")
    d.close()


def _oracle_each(jobs, threads=None):
    """oracle.run on independent (geometry, hits, t0) jobs, one slice per
    call, spread over the host cores (the oracle's C code runs without the
    interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as orc

    def one(job):
        g, par, hits, t0 = job
        return orc.run(g.xyz_mm, g.floor_id, par, hits, [t0], threads=1)[0]

    with ThreadPoolExecutor(threads or os.cpu_count() or 4) as ex:
        return list(ex.map(one, jobs))


def test_batched_config_all_slices(pkg, params):
    """The headline workload: all 64 slices in one launch sequence (graph
    replay), every slice compared with the oracle element by element.  The
    slices are independent runs (no halos), so each gets its own oracle
    call."""
    wl = workload.cfg_batched()
    dets = [_det(pkg, g, params) for g in wl.detectors]
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    b = DeviceBatch([SliceIn(dets[s.det_index], s.t0, s.stream.hits, s.stream.pmt_off) for s in wl.submissions])
    b.run(graph=True)
    b.run(graph=True)                   # the replay, as the bench times it
    res = b.results()
    refs = _oracle_each([(wl.detectors[s.det_index], params, s.stream.hits, s.t0) for s in wl.submissions])
    assert len(res) == len(refs) == 64
    for k, (r, ref) in enumerate(zip(res, refs)):
        _assert_same(r, ref, f"batched slice {k}")
    for d in dets:
        d.close()


# ---------------------------------------------------------- tiles and edges

def test_result_independent_of_tile_configuration(pkg, params):
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    subs = [(s.t0, s.stream) for s in wl.submissions[:2]]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0][:2])
    old = pkg.trig_get_tile_config()
    try:
        for cap, warps, fill in ((1024, 4, 40), (1024, 4, 85), (2048, 8, 30), (2048, 8, 90), (2048, 16, 60), (4096, 8, 50), (4096, 16, 15), (4096, 16, 60),
                                 (4096, 16, 95)):
            pkg.trig_set_tile_config(cap, warps, fill)
            _, res = _run(pkg, d, subs)
            for k in range(2):
                _assert_same(res[k], ref[k], f"cap {cap} warps {warps} fill {fill} slice {k}")
    finally:
        pkg.trig_set_tile_config(*old)
    d.close()


def test_autotuned_shape_keeps_results(pkg, params, tmp_path, monkeypatch):
    """The autotuner picks a launch shape per detector and records it in the
    cache file; results stay exact under the chosen shape, and a new
    detector of the same size picks the cached shape up."""
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TRIG_TUNE_CACHE", str(cache))
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    b = DeviceBatch([SliceIn(d, s.t0, s.stream.hits, s.stream.pmt_off) for s in wl.submissions[:3]])
    r = pkg.trig_autotune(d, b.descs)
    assert r["n_tried"] == 20 and r["ms"] > 0
    assert pkg.trig_detector_tile_config(d) == dict(cap=r["cap"], warps=r["warps"], fill_pct=r["fill_pct"], tuned=True)
    b.run(graph=True)
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0][:3])
    for k, res in enumerate(b.results()):
        _assert_same(res, ref[k], f"tuned slice {k}")
    line = cache.read_text().split()
    assert int(line[1]) == g.n_pmt and int(line[2]) == r["cap"] and int(line[3]) == r["warps"]
    d2 = _det(pkg, g, params)
    assert pkg.trig_detector_tile_config(d2)["tuned"]
    d.close()
    d2.close()


def test_dense_burst_takes_split_path(pkg, params):
    """A burst far above the tile's planned density: tiles overflow and
    are split; results stay exact."""
    g = workload.nemo_tower()
    par = dict(params, slice_ns=2_000_000)
    t0 = workload.T_ORIGIN_NS
    st = workload.gen_stream(g, t0 - 3000, t0 + par["slice_ns"] + 3000, 50e3, seed=3, stream=1)
    rng = np.random.Generator(np.random.PCG64(9))
    burst = np.zeros(30_000, workload.HIT_DTYPE)
    burst["t"] = rng.integers(t0 + 700_000, t0 + 760_000, len(burst))
    burst["pmt"] = rng.integers(0, 32, len(burst))
    burst["charge"] = rng.integers(50, 400, len(burst))
    hits = np.concatenate([st.hits, burst])
    full = _stream_from_hits(hits, g.n_pmt)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, [(t0, full)])
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, [t0])
    _assert_same(res[0], ref[0], "burst")
    d.close()


def test_degenerate_single_ns_pileup_reports_capacity(pkg, params):
    g = workload.nemo_tower()
    par = dict(params, slice_ns=1_000_000)
    t0 = 10_000_000
    hits = np.zeros(6000, workload.HIT_DTYPE)
    hits["t"] = t0 + 5000
    hits["pmt"] = np.arange(6000) % 32
    hits["charge"] = 100
    full = _stream_from_hits(hits, g.n_pmt)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, [(t0, full)])
    stats = res[0][0]
    assert int(stats["status"]) == pkg.TRIG_ECAPACITY
    assert int(stats["flags"]) & 0x08
    d.close()


def test_edge_cases_empty_and_single(pkg, params):
    g = workload.nemo_tower()
    d = _det(pkg, g, params)
    t0 = 10_000_000
    empty = workload.Stream(np.zeros(0, workload.HIT_DTYPE), np.zeros(33, np.uint64))
    one = np.zeros(1, workload.HIT_DTYPE)
    one["t"], one["pmt"], one["charge"] = t0, 5, 500
    only_halo = np.zeros(2, workload.HIT_DTYPE)
    only_halo["t"], only_halo["pmt"], only_halo["charge"] = [t0 - 100, t0 - 90], [0, 1], 100
    subs = [(t0, empty), (t0, _stream_from_hits(one, 32)), (t0, _stream_from_hits(only_halo, 32))]
    _, res = _run(pkg, [d, d, d], subs)
    assert int(res[0][0]["status"]) == 0 and len(res[0][1]) == 0 and int(res[0][0]["n_seeds"]) == 0
    assert int(res[1][0]["n_seeds"]) == 1 and len(res[1][1]) == 0
    assert int(res[2][0]["n_seeds"]) == 0 and len(res[2][1]) == 0
    d.close()


def test_malformed_input_is_flagged(pkg, params):
    g = workload.nemo_tower()
    d = _det(pkg, g, params)
    t0 = 10_000_000
    h = np.zeros(3, workload.HIT_DTYPE)
    h["t"] = [t0 + 10, t0 + 5, t0 + 20]
    h["pmt"] = [3, 3, 3]
    off = np.zeros(33, np.uint64)
    off[4:] = 3
    unsorted = workload.Stream(h, off)
    h2 = h.copy()
    h2["t"] = [t0, t0 + 1, t0 + 2]
    h2["pmt"] = [3, 7, 3]
    wrong_row = workload.Stream(h2, off)
    h3 = h2.copy()
    h3["pmt"] = 3
    h3["t"] = [t0, t0 + 1, t0 + params["slice_ns"] + 3000]
    out_of_range = workload.Stream(h3, off)
    _, res = _run(pkg, [d, d, d], [(t0, unsorted), (t0, wrong_row), (t0, out_of_range)])
    assert int(res[0][0]["status"]) == pkg.TRIG_EINVAL and int(res[0][0]["flags"]) & 0x02
    assert int(res[1][0]["status"]) == pkg.TRIG_EINVAL and int(res[1][0]["flags"]) & 0x01
    assert int(res[2][0]["status"]) == pkg.TRIG_EINVAL and int(res[2][0]["flags"]) & 0x04
    d.close()


def test_output_capacity_flag(pkg, params):
    wl = workload.cfg_nemo()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    s = wl.submissions[0]
    b = DeviceBatch([SliceIn(d, s.t0, s.stream.hits, s.stream.pmt_off)], trig_cap=10)
    b.run()
    stats, trig, win = b.results()[0]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])[0]
    assert int(stats["status"]) == pkg.TRIG_ECAPACITY
    assert int(stats["n_triggers"]) == len(ref.triggers)
    assert len(trig) == 10
    assert np.array_equal(trig["t"], ref.triggers["t"][:10])
    d.close()


# ------------------------------------------------------------ wide detectors

def _tower_array(nx, ny):
    return workload.tower_array(nx=nx, ny=ny)


@pytest.mark.parametrize("nx,ny,rate,seed", [(2, 1, 200e3, 1), (4, 2, 55e3, 2), (3, 3, 120e3, 3)])
def test_wide_detector_slices(pkg, params, nx, ny, rate, seed):
    """Detectors with 168..756 PMTs take the bucketed staging path; three
    contiguous slices with halos and injected muons, exact against the
    oracle, in one batch, per slice and as a graph replay."""
    g = _tower_array(nx, ny)
    assert g.n_pmt >= 129
    par = dict(params, slice_ns=3_000_000)
    t0 = workload.T_ORIGIN_NS
    t0s = [t0 + k * par["slice_ns"] for k in range(3)]
    full = workload.gen_stream(g, t0 - 3000, t0s[-1] + par["slice_ns"] + 3000, rate, n_muons=40, seed=seed,
                               stream=70 + seed)
    d = _det(pkg, g, par)
    subs = _subs_from_run(full, t0s, par["slice_ns"])
    ref = oracle.run(g.xyz_mm, g.floor_id, par, full.hits, t0s)
    for mode in ("batch", "each", "graph"):
        _, res = _run(pkg, d, subs, graph=mode == "graph", each=mode == "each")
        for k in range(3):
            _assert_same(res[k], ref[k], f"{g.n_pmt} PMTs {mode} slice {k}")
    d.close()


def test_wide_detector_burst_and_row_outputs(pkg, params):
    """A dense burst on a wide detector overflows its bucketed tiles (split
    path); the merged rows and seed counts match the oracle row by row."""
    g = _tower_array(2, 1)
    par = dict(params, slice_ns=1_000_000)
    t0 = workload.T_ORIGIN_NS
    st = workload.gen_stream(g, t0 - 3000, t0 + par["slice_ns"] + 3000, 80e3, seed=5, stream=90)
    rng = np.random.Generator(np.random.PCG64(11))
    burst = np.zeros(20_000, workload.HIT_DTYPE)
    burst["t"] = rng.integers(t0 + 400_000, t0 + 430_000, len(burst))
    burst["pmt"] = rng.integers(0, g.n_pmt, len(burst))
    burst["charge"] = rng.integers(50, 400, len(burst))
    hits = np.concatenate([st.hits, burst])
    full = _stream_from_hits(hits, g.n_pmt)
    d = _det(pkg, g, par)
    b, res = _run(pkg, d, [(t0, full)])
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, [t0])
    _assert_same(res[0], ref[0], "wide burst")
    merged, seedcnt = b.rows(0)
    own = hits[(hits["t"] >= t0) & (hits["t"] < t0 + par["slice_ns"])]
    om = oracle.merge(own)
    for f in ("t", "pmt", "charge"):
        assert np.array_equal(merged[f], om[f]), f
    is_seed = seedcnt != 0xFFFFFFFF
    assert np.array_equal(merged["t"][is_seed], ref[0].seeds["t"])
    assert np.array_equal(seedcnt[is_seed], ref[0].seeds["count"])
    d.close()


# ------------------------------------------------------------ event payload

def _events_run(pkg, det, subs, graph=False):
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    b = DeviceBatch([SliceIn(det if not isinstance(det, list) else det[i], t0, s.hits, s.pmt_off)
                     for i, (t0, s) in enumerate(subs)], events=True)
    b.run(graph=graph)
    return b.results(), b.event_hits()


def _assert_events(ev_res, ref_hits, ref_windows, ctx):
    ev, ne, full = ev_res
    want = oracle.events(ref_hits, ref_windows)
    assert not full, ctx
    assert ne == len(want) == int(ref_windows["n_hits"].sum()), (ctx, ne, len(want))
    for f in ("t", "pmt", "charge"):
        assert np.array_equal(ev[f], want[f]), (ctx, f)


@pytest.mark.parametrize("graph", [False, True])
def test_events_km3_five_slices(pkg, params, graph):
    """The hits inside the merged windows of five contiguous KM3Net-It
    slices (with bursts), in merged order, halos included."""
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    res, evs = _events_run(pkg, d, [(s.t0, s.stream) for s in wl.submissions], graph=graph)
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])
    for k in range(len(ref)):
        _assert_same(res[k], ref[k], f"km3 slice {k}")
        _assert_events(evs[k], wl.runs[0].hits, ref[k].windows, f"km3 events {k}")
    d.close()


def test_events_nemo_and_wide_detector(pkg, params):
    for g, rate, slice_ns in ((workload.nemo_tower(), 50e3, 200_000_000), (_tower_array(3, 1), 150e3, 4_000_000)):
        par = dict(params, slice_ns=slice_ns)
        t0 = workload.T_ORIGIN_NS
        t0s = [t0, t0 + slice_ns]
        full = workload.gen_stream(g, t0 - 3000, t0 + 2 * slice_ns + 3000, rate, n_muons=30, seed=4, stream=120)
        d = _det(pkg, g, par)
        res, evs = _events_run(pkg, d, _subs_from_run(full, t0s, slice_ns))
        ref = oracle.run(g.xyz_mm, g.floor_id, par, full.hits, t0s)
        for k in range(2):
            _assert_same(res[k], ref[k], f"{g.n_pmt} slice {k}")
            _assert_events(evs[k], full.hits, ref[k].windows, f"{g.n_pmt} events {k}")
        d.close()


def test_events_capacity_flag(pkg, params):
    """An event buffer smaller than the payload: TRIG_FLAG_EV_FULL, status
    ECAPACITY, n_events still counted, triggers and windows unaffected."""
    import torch
    from paper_1411_3968_gb300 import _lib
    from paper_1411_3968_gb300.runner import DeviceBatch, SliceIn
    wl = workload.cfg_nemo()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    s = wl.submissions[0]
    b = DeviceBatch([SliceIn(d, s.t0, s.stream.hits, s.stream.pmt_off)], events=True)
    b.events[0] = _lib.trig_slice_events(b.ev[0].data_ptr(), 10)
    b.ev_cap[0] = 10
    b.ensure_scratch()
    b.run()
    stats, trig, win = b.results()[0]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])[0]
    assert int(stats["status"]) == pkg.TRIG_ECAPACITY and int(stats["flags"]) & _lib.TRIG_FLAG_EV_FULL
    assert int(stats["n_events"]) == int(ref.windows["n_hits"].sum())
    assert np.array_equal(trig["t"], ref.triggers["t"]) and np.array_equal(win["n_hits"], ref.windows["n_hits"])
    d.close()


# ------------------------------------------------------------------ level 0

@pytest.mark.parametrize("distinct", [0, 1])
def test_level0_towers(pkg, params, distinct):
    """N7TW1000 (and its distinct-PMT form) before the seed triggers, on
    the KM3Net-It run with bursts and the NEMO slice: exact against the
    oracle."""
    for wl in (workload.cfg_km3(), workload.cfg_nemo()):
        g = wl.detectors[0]
        par = dict(params, l0_hits=7, l0_window_ns=1000, l0_distinct_pmts=distinct)
        d = _det(pkg, g, par)
        _, res = _run(pkg, d, [(s.t0, s.stream) for s in wl.submissions])
        ref = oracle.run(g.xyz_mm, g.floor_id, par, wl.runs[0].hits, wl.run_slices[0])
        for k in range(len(ref)):
            _assert_same(res[k], ref[k], f"{g.name} level0 distinct={distinct} slice {k}")
        d.close()


@pytest.mark.parametrize("case", range(6))
def test_level0_random_dense(pkg, params, case):
    rng = np.random.Generator(np.random.PCG64(900 + case))
    g = [workload.nemo_tower, workload.km3_tower][case % 2]()
    par = dict(params, slice_ns=int(rng.choice([20_000, 200_000])), threshold=int(rng.integers(1, 5)),
               l0_hits=int(rng.integers(2, 9)), l0_window_ns=int(rng.choice([30, 300, 1000, 4000])),
               l0_distinct_pmts=int(case % 3 == 0))
    t0 = 5_000_000
    n = int(rng.integers(300, 3000))
    t = rng.integers(t0 - 4000, t0 + 2 * par["slice_ns"] + 4000, n)
    t[: n // 3] = t[n // 3: 2 * (n // 3)] + rng.integers(-200, 201, n // 3)
    hits = np.zeros(n, workload.HIT_DTYPE)
    hits["t"] = t
    hits["pmt"] = rng.integers(0, g.n_pmt, n)
    hits["charge"] = rng.integers(1, 500, n)
    t0s = [t0, t0 + par["slice_ns"]]
    full = _stream_from_hits(hits, g.n_pmt)
    d = _det(pkg, g, par)
    halo = d.halo_ns
    _, res = _run(pkg, d, _subs_from_run(full, t0s, par["slice_ns"], halo))
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, t0s)
    for k in range(2):
        _assert_same(res[k], ref[k], f"case {case} slice {k}")
    d.close()


def test_level0_wide_detector(pkg, params):
    g = _tower_array(3, 1)
    par = dict(params, slice_ns=2_000_000, l0_hits=10, l0_window_ns=800)
    t0 = workload.T_ORIGIN_NS
    t0s = [t0, t0 + par["slice_ns"]]
    full = workload.gen_stream(g, t0 - 3000, t0 + 2 * par["slice_ns"] + 3000, 120e3, n_muons=30, seed=8, stream=140)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, _subs_from_run(full, t0s, par["slice_ns"]))
    ref = oracle.run(g.xyz_mm, g.floor_id, par, full.hits, t0s)
    for k in range(2):
        _assert_same(res[k], ref[k], f"wide level0 slice {k}")
    d.close()


def test_distinct_level0_above_128_pmts(pkg, params):
    """DN7TW1000 (level 0 over different PMTs) on a 168-PMT two-tower array
    and on the 2688-PMT array (a warp per seed with a shared-memory PMT set):
    exact against the oracle on two contiguous slices each."""
    for g, rate, slice_ns, n_req in ((_tower_array(2, 1), 300e3, 500_000, 48),
                                     (_tower_array(8, 4), 55e3, 200_000, 150)):
        par = dict(params, slice_ns=slice_ns, l0_hits=n_req, l0_window_ns=1000, l0_distinct_pmts=1)
        t0 = workload.T_ORIGIN_NS
        t0s = [t0, t0 + slice_ns]
        full = workload.gen_stream(g, t0 - 3000, t0 + 2 * slice_ns + 3000, rate, n_muons=20, seed=10, stream=160)
        d = _det(pkg, g, par)
        _, res = _run(pkg, d, _subs_from_run(full, t0s, slice_ns))
        ref = oracle.run(g.xyz_mm, g.floor_id, par, full.hits, t0s)
        off = oracle.run(g.xyz_mm, g.floor_id, dict(par, l0_hits=0), full.hits, t0s)
        assert sum(len(r.seeds) for r in ref) > 0
        assert sum(len(r.seeds) for r in ref) < sum(len(r.seeds) for r in off)     # level 0 drops seeds
        for k in range(2):
            _assert_same(res[k], ref[k], f"distinct level 0, {g.n_pmt} PMTs, slice {k}")
        d.close()


def test_level0_parameter_checks(pkg, params):
    with pytest.raises(pkg.TrigError):
        _det(pkg, workload.nemo_tower(), dict(params, l0_hits=7, l0_window_ns=0))


# ------------------------------------------- coincidence ladder, distinct count

LADDER = dict(seed_rule=1, threshold=1)


@pytest.mark.parametrize("variant", ["ladder", "ladder_n7tw", "ladder_c4", "distinct", "distinct_ladder"])
def test_rule_variants_towers(pkg, params, variant):
    """The paper's coincidence ladder ([SC and AFC] or [FC and AFC], alone,
    after N7TW1000, or followed by the causal count at 4) and the
    distinct-PMT causal count, on the KM3Net-It run with bursts and on the
    NEMO slice: exact against the oracle."""
    extra = {"ladder": LADDER, "ladder_n7tw": dict(LADDER, l0_hits=7, l0_window_ns=1000),
             "ladder_c4": dict(seed_rule=1), "distinct": dict(count_distinct_pmts=1),
             "distinct_ladder": dict(LADDER, count_distinct_pmts=1, threshold=3)}[variant]
    for wl in (workload.cfg_km3(), workload.cfg_nemo()):
        g = wl.detectors[0]
        par = dict(params, **extra)
        d = _det(pkg, g, par)
        _, res = _run(pkg, d, [(s.t0, s.stream) for s in wl.submissions])
        ref = oracle.run(g.xyz_mm, g.floor_id, par, wl.runs[0].hits, wl.run_slices[0], tower_id=g.tower_id)
        assert sum(len(r.seeds) for r in ref) > 0, variant
        for k in range(len(ref)):
            _assert_same(res[k], ref[k], f"{g.name} {variant} slice {k}")
        d.close()


@pytest.mark.parametrize("case", range(6))
def test_rule_variants_random_dense(pkg, params, case):
    """Dense random slices with clustered coincidences, several tile
    widths' worth of hits: random windows, distances and thresholds."""
    rng = np.random.Generator(np.random.PCG64(950 + case))
    g = [workload.nemo_tower, workload.km3_tower][case % 2]()
    par = dict(params, slice_ns=int(rng.choice([20_000, 200_000])), seed_rule=int(case % 3 != 2),
               threshold=int(rng.integers(1, 4)), count_distinct_pmts=int(case % 2 == 0),
               sc_window_ns=int(rng.choice([20, 60])), fc_window_ns=int(rng.choice([10, 100])),
               afc_window_ns=int(rng.choice([100, 250, 700])), sc_dist_mm=int(rng.choice([1000, 7000])))
    t0 = 5_000_000
    n = int(rng.integers(1500, 5000))
    t = rng.integers(t0 - 4000, t0 + 2 * par["slice_ns"] + 4000, n)
    t[: n // 2] = t[n // 2: 2 * (n // 2)] + rng.integers(-300, 301, n // 2)
    hits = np.zeros(n, workload.HIT_DTYPE)
    hits["t"] = t
    hits["pmt"] = rng.integers(0, g.n_pmt, n)
    hits["charge"] = rng.integers(1, 500, n)
    t0s = [t0, t0 + par["slice_ns"]]
    full = _stream_from_hits(hits, g.n_pmt)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, _subs_from_run(full, t0s, par["slice_ns"], d.halo_ns))
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, t0s, tower_id=g.tower_id)
    assert sum(len(r.seeds) for r in ref) > 0
    for k in range(2):
        _assert_same(res[k], ref[k], f"case {case} slice {k}")
    d.close()


def test_ladder_wide_detector_with_towers(pkg, params):
    """A 3 x 1 tower array (252 PMTs, bucketed staging): the consecutive-
    floor test uses the tower ids."""
    g = _tower_array(3, 1)
    par = dict(params, slice_ns=2_000_000, seed_rule=1, threshold=2)
    t0 = workload.T_ORIGIN_NS
    t0s = [t0, t0 + par["slice_ns"]]
    full = workload.gen_stream(g, t0 - 3000, t0 + 2 * par["slice_ns"] + 3000, 150e3, n_muons=40, seed=9, stream=141)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, _subs_from_run(full, t0s, par["slice_ns"]))
    ref = oracle.run(g.xyz_mm, g.floor_id, par, full.hits, t0s, tower_id=g.tower_id)
    assert sum(len(r.seeds) for r in ref) > 0
    for k in range(2):
        _assert_same(res[k], ref[k], f"wide ladder slice {k}")
    d.close()


def test_distinct_count_above_128_pmts(pkg, params):
    """The distinct-PMT count on a 168-PMT two-tower array and on the
    2688-PMT array (a warp per seed with a shared-memory PMT set): exact
    against the oracle on two contiguous slices each."""
    for g, rate, slice_ns in ((_tower_array(2, 1), 150e3, 1_000_000), (_tower_array(8, 4), 55e3, 200_000)):
        par = dict(params, slice_ns=slice_ns, count_distinct_pmts=1)
        t0 = workload.T_ORIGIN_NS
        t0s = [t0, t0 + slice_ns]
        full = workload.gen_stream(g, t0 - 3000, t0 + 2 * slice_ns + 3000, rate, n_muons=20, seed=9, stream=150)
        d = _det(pkg, g, par)
        _, res = _run(pkg, d, _subs_from_run(full, t0s, slice_ns))
        ref = oracle.run(g.xyz_mm, g.floor_id, par, full.hits, t0s)
        assert sum(len(r.triggers) for r in ref) > 0
        for k in range(2):
            _assert_same(res[k], ref[k], f"distinct count, {g.n_pmt} PMTs, slice {k}")
        d.close()


def test_rule_parameter_checks(pkg, params):
    with pytest.raises(pkg.TrigError):
        _det(pkg, workload.nemo_tower(), dict(params, seed_rule=2))
    with pytest.raises(pkg.TrigError):
        _det(pkg, workload.nemo_tower(), dict(params, seed_rule=1, afc_window_ns=60001))


# ------------------------------------------------------ multi-tower selection

def _array_oracle(wl, par, K, W, h, k=0):
    import oracle.array as oa
    nt = len(wl.detectors)
    seeds = [oracle.run(g.xyz_mm, g.floor_id, par, wl.runs[b].hits, [wl.run_slices[b][k]])[0].triggers
             for b, g in enumerate(wl.detectors)]
    return oa.select([g.xyz_mm for g in wl.detectors], par, K, W, h, seeds,
                     [(wl.runs[b].hits, wl.runs[b].pmt_off) for b in range(nt)])


def _array_run(pkg, wl, par, K, W, h, k=0, graph=False, **caps):
    from paper_1411_3968_gb300.runner import ArrayBatch, SliceIn
    nt = len(wl.detectors)
    dets = [_det(pkg, g, par) for g in wl.detectors]
    arr = pkg.Array(dets, min_towers=K, corr_window_ns=W, win_half_ns=h)
    subs = wl.submissions[k * nt:(k + 1) * nt]
    ab = ArrayBatch(arr, [SliceIn(dets[s.det_index], s.t0, s.stream.hits, s.stream.pmt_off) for s in subs], **caps)
    ab.run(graph=graph)
    out = ab.results()
    return out, (ab, arr, dets)


def _assert_array_same(got, ref, ctx=""):
    st, seeds, wins, frag, hits = got
    assert int(st["status"]) == 0 and int(st["flags"]) == 0, (ctx, st)
    assert int(st["n_selected"]) == len(ref.seeds), ctx
    for f in ("t", "pmt", "tower", "n_towers"):
        assert np.array_equal(seeds[f], ref.seeds[f]), (ctx, f)
    assert len(wins) == len(ref.windows), ctx
    for f in ("lo", "hi", "n_hits", "n_triggers"):
        assert np.array_equal(wins[f], ref.windows[f]), (ctx, f)
    assert np.array_equal(frag, ref.frag_off), ctx
    for f in ("t", "pmt", "charge"):
        assert np.array_equal(hits[f], ref.hits[f]), (ctx, f)


@pytest.mark.parametrize("K,W,h", [(2, 3000, 3000), (1, 3000, 3000), (3, 3000, 2000), (2, 800, 3000)])
def test_array_selection_towers8(pkg, params, K, W, h):
    """The eight KM3Net-It towers, one 200 ms slice each: selected seeds,
    merged windows, fragment offsets and the readback, exact against the
    oracle."""
    wl = workload.cfg_towers8()
    got, keep = _array_run(pkg, wl, params, K, W, h)
    ref = _array_oracle(wl, params, K, W, h)
    assert len(ref.seeds) > 0
    _assert_array_same(got, ref, f"K={K} W={W} h={h}")


def test_array_selection_two_slices_graph(pkg, params):
    """Two contiguous periods (each tower's submission carries its halos),
    the towers' trigger as a graph replay before the selection."""
    wl = workload.cfg_towers8(seed=3, n_slices=2)
    for k in range(2):
        got, keep = _array_run(pkg, wl, params, 2, 3000, 3000, k=k, graph=True)
        _assert_array_same(got, _array_oracle(wl, params, 2, 3000, 3000, k=k), f"period {k}")


def test_array_selection_capacity_flags(pkg, params):
    """Outputs smaller than needed: the flags say so and what was stored is
    the prefix of the full result."""
    wl = workload.cfg_towers8()
    ref = _array_oracle(wl, params, 2, 3000, 3000)
    nw = max(1, len(ref.windows) // 2)
    (st, seeds, wins, frag, hits), keep = _array_run(pkg, wl, params, 2, 3000, 3000, seed_cap=5, win_cap=nw,
                                                      hit_cap=10)
    assert st["flags"] & pkg.TRIG_AFLAG_SEED_FULL and st["flags"] & pkg.TRIG_AFLAG_WIN_FULL
    assert st["flags"] & pkg.TRIG_AFLAG_HIT_FULL and int(st["status"]) == pkg.TRIG_ECAPACITY
    assert int(st["n_selected"]) == len(ref.seeds) and int(st["n_windows"]) == len(ref.windows)
    assert np.array_equal(seeds["t"], ref.seeds["t"][:5])
    assert np.array_equal(wins["lo"], ref.windows["lo"][:nw])
    assert np.array_equal(frag, ref.frag_off[: nw * 8 + 1])
    assert np.array_equal(hits["t"], ref.hits["t"][:10])


def test_array_golden_fixture_on_gpu(pkg, params):
    """The hand-derived two-tower fixture through the CUDA path."""
    import json
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "array", "two_towers.json")))
    from paper_1411_3968_gb300.runner import ArrayBatch, SliceIn
    t0 = fx["t0"]
    towers = workload.split_towers(workload.tower_array(nx=2, ny=1))
    par = dict(params, **fx["tower_params"])
    streams = [workload.stream_from_rows([(t0 + t, p, q) for (t, p, q) in rows], 84) for rows in fx["hits_rel"]]
    dets = [_det(pkg, g, par) for g in towers]
    for name, v in fx["variants"].items():
        ap = dict(fx["array_params"], **v["array_params"])
        arr = pkg.Array(dets, **ap)
        ab = ArrayBatch(arr, [SliceIn(d, t0, st.hits, st.pmt_off) for d, st in zip(dets, streams)])
        ab.run()
        st, seeds, wins, frag, hits = ab.results()
        assert int(st["status"]) == 0, name
        assert [[int(s["t"]) - t0, int(s["pmt"]), int(s["tower"]), int(s["n_towers"])] for s in seeds] == \
            v["seeds_rel"], name
        assert [[int(w["lo"]) - t0, int(w["hi"]) - t0, int(w["n_hits"]), int(w["n_triggers"])] for w in wins] == \
            v["windows_rel"], name
        frags = [[[int(x["t"]) - t0, int(x["pmt"]), int(x["charge"])] for x in hits[int(a):int(b)]]
                 for a, b in zip(frag[:-1], frag[1:])]
        assert frags == v["fragments_rel"], name
        del ab
        arr.close()


def test_array_parameter_checks(pkg, params):
    towers = workload.split_towers(workload.tower_array(nx=2, ny=1))
    dets = [_det(pkg, g, params) for g in towers]
    with pytest.raises(pkg.TrigError):
        pkg.Array(dets, min_towers=0)
    with pytest.raises(pkg.TrigError):
        pkg.Array(dets, win_half_ns=4000)                   # beyond the towers' 3000 ns halo
    odd = _det(pkg, towers[1], dict(params, tol_ns=25))
    with pytest.raises(pkg.TrigError):
        pkg.Array([dets[0], odd])


def test_sparse_and_dense_count_builds_agree(pkg, params):
    """A tower slice alone runs the 4-lanes-per-seed build; batched with the
    dense 2688-PMT slice it runs the warp-per-seed build.  Both equal the
    oracle."""
    wl = workload.cfg_nemo()
    g = wl.detectors[0]
    d = _det(pkg, g, params)
    s = wl.submissions[0]
    ref = oracle.run(g.xyz_mm, g.floor_id, params, wl.runs[0].hits, wl.run_slices[0])[0]
    _, alone = _run(pkg, d, [(s.t0, s.stream)])
    _assert_same(alone[0], ref, "sparse build")
    arr = _tower_array(8, 4)
    da = _det(pkg, arr, params)
    t0 = workload.T_ORIGIN_NS + 10 * params["slice_ns"]
    st = workload.gen_stream(arr, t0 - 3000, t0 + params["slice_ns"] + 3000, 55e3, n_muons=20, seed=12, stream=150)
    _, both = _run(pkg, [d, da], [(s.t0, s.stream), (t0, st)])
    _assert_same(both[0], ref, "dense build")
    d.close()
    da.close()


@pytest.mark.parametrize("n", [31, 32, 33, 511, 512, 513, 4095, 4096, 4097, 9000])
def test_structure_pass_walk_edges(pkg, params, n):
    """Hit counts around the structure pass's warp range (512) and chunk
    (4096); PMT runs that start or end a warp range; only the first, only
    the last, or a single PMT populated: results equal the oracle."""
    g = workload.km3_tower()
    rng = np.random.Generator(np.random.PCG64(2000 + n))
    par = dict(params, slice_ns=20_000)
    t0 = 7_000_000
    for layout in ("mixed", "first", "last", "single"):
        if layout == "mixed":
            pmts = rng.integers(0, g.n_pmt, n)
        elif layout == "first":
            pmts = np.zeros(n, np.int64)
        elif layout == "last":
            pmts = np.full(n, g.n_pmt - 1)
        else:
            pmts = np.full(n, 40)
        hits = np.zeros(n, workload.HIT_DTYPE)
        hits["t"] = rng.integers(t0, t0 + par["slice_ns"], n)
        hits["pmt"] = pmts
        hits["charge"] = rng.integers(1, 500, n)
        d = _det(pkg, g, par)
        _, res = _run(pkg, d, [(t0, _stream_from_hits(hits, g.n_pmt))])
        ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, [t0])[0]
        _assert_same(res[0], ref, f"n={n} {layout}")
        d.close()


def test_array_selection_with_an_empty_tower(pkg, params):
    """One tower submits no hits (no triggers, empty fragments) and another
    only background far below threshold: selection and readback equal the
    oracle, with K = 2 and K = 1."""
    wl = workload.cfg_towers8(seed=5)
    nt = len(wl.detectors)
    subs = list(wl.submissions[:nt])
    runs = list(wl.runs)
    empty = workload.Stream(np.zeros(0, workload.HIT_DTYPE), np.zeros(85, np.uint64))
    subs[3] = workload.Submission(3, subs[3].t0, empty)
    runs[3] = empty
    wl2 = workload.Workload("towers8_empty3", wl.detectors, subs, runs, wl.run_slices)
    for K in (2, 1):
        got, keep = _array_run(pkg, wl2, params, K, 3000, 3000)
        ref = _array_oracle(wl2, params, K, 3000, 3000)
        _assert_array_same(got, ref, f"empty tower K={K}")
        assert not (ref.seeds["tower"] == 3).any()


def test_maximum_pmt_count(pkg, params):
    """A detector at the 4096-PMT limit (512 floors of 8 PMTs scattered in a
    1 km box): the wide path with the largest dt table, exact against the
    oracle; one PMT more is refused."""
    rng = np.random.Generator(np.random.PCG64(4096))
    P = 4096
    xyz = rng.integers(-500_000, 500_000, (P, 3)).astype(np.int32)
    floor = (np.arange(P) // 8).astype(np.uint32)
    xyz[:, 2] = (floor.astype(np.int64) * 2000 - 500_000).astype(np.int32)    # floors stacked 2 m apart
    g = workload.Detector("max4096", xyz, floor, np.zeros(P, np.uint32))
    # most pairs sit beyond the 3 us clamp, so counts run near 300: a
    # threshold of 330 fires about a fifth of the seeds in 30 windows
    par = dict(params, slice_ns=1_000_000, threshold=330)
    t0 = 50_000_000
    n = 60_000
    hits = np.zeros(n, workload.HIT_DTYPE)
    hits["t"] = rng.integers(t0 - 3000, t0 + par["slice_ns"] + 3000, n)
    hits["t"][: n // 4] = hits["t"][n // 4: n // 2] + rng.integers(-15, 16, n // 4)
    hits["t"] = np.clip(hits["t"], t0 - 3000, t0 + par["slice_ns"] + 2999)     # inside the accepted halos
    hits["pmt"] = rng.integers(0, P, n)
    hits["pmt"][: n // 4] = (hits["pmt"][n // 4: n // 2] // 8) * 8 + rng.integers(0, 8, n // 4)
    hits["charge"] = rng.integers(1, 500, n)
    d = _det(pkg, g, par)
    _, res = _run(pkg, d, [(t0, _stream_from_hits(hits, P))])
    ref = oracle.run(g.xyz_mm, g.floor_id, par, hits, [t0])[0]
    assert 0 < len(ref.triggers) < len(ref.seeds) and len(ref.windows) > 1
    _assert_same(res[0], ref, "4096 PMTs")
    d.close()
    with pytest.raises(pkg.TrigError):
        pkg.Detector(np.zeros((P + 1, 3), np.int32), np.zeros(P + 1, np.uint32), params)
