"""Pins of the CPU oracle against things other than itself.

* hand-derived golden fixtures (tests/golden/*.json, each with its citation
  and the derivation of every expected value);
* the exact-integer dt_max against independent big-integer arithmetic and
  against ceil() in extended precision on random distances;
* an independent all-pairs brute force (no sort, no window, pure Python)
  on tiny random slices with forced ties and coincidences;
* closed forms on pure Poisson background: the accidental floor-coincidence
  seed rate and the mean causal count;
* recovery of every injected muon track that fires on its own hits;
* invariance of the triggers under a different partition of the run.
"""
import glob
import json
import math
import os

import numpy as np
import pytest

import oracle
import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GEOMETRIES = {"nemo32": workload.nemo_tower, "km3it84": workload.km3_tower, "array2688": workload.tower_array}


def _tuples(a, fields):
    return [tuple(int(x[f]) for f in fields) for x in a]


SEED_F = ("t", "pmt", "charge", "count")
WIN_F = ("lo", "hi", "n_hits", "n_triggers")


# ------------------------------------------------------------------ golden

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))), ids=os.path.basename)
def test_golden_fixture(path, params):
    fx = json.load(open(path))
    det = GEOMETRIES[fx["geometry"]]()
    par = dict(params)
    par.update(fx["params"])
    hits = np.zeros(len(fx["hits"]), oracle.HIT_DTYPE)
    for i, (t, p, q) in enumerate(fx["hits"]):
        hits[i] = (t, p, q, 0)
    res = oracle.run(det.xyz_mm, det.floor_id, par, hits, fx["slices"])
    for r, exp in zip(res, fx["expected"]):
        assert _tuples(r.seeds, SEED_F) == [tuple(x) for x in exp["seeds"]]
        assert _tuples(r.triggers, SEED_F) == [tuple(x) for x in exp["triggers"]]
        assert _tuples(r.windows, WIN_F) == [tuple(x) for x in exp["windows"]]


# ------------------------------------------------------------------ dt_max

def _k_exact(d2, n_num=6900, n_den=1499):
    """Smallest k with k * n_den * 1000 >= n_num * sqrt(d2): integer square
    root on Python big integers (independent of the oracle's search)."""
    M = n_den * 1000
    X = n_num * n_num * d2
    r = math.isqrt(X)
    if r * r == X:
        return (r + M - 1) // M
    return r // M + 1


def test_dtmax_worked_values():
    # distances in mm, expected dt_max by hand: 20 + ceil(d[m] * 1.38 / 0.2998)
    cases = {
        0: 20,                                   # same point
        6000 ** 2: 48,                           # across a 6 m bar: ceil(27.62) = 28
        40000 ** 2: 205,                         # one floor straight up: ceil(184.12) = 185
        1618 * 10 ** 6: 206,                     # rotated adjacent floor, sqrt(1618) m
        80000 ** 2: 389,                         # two floors up: ceil(368.25)
        14990 ** 2: 89,                          # 14.99 m: exactly 69, ceil of an integer
        14990 ** 2 + 1: 90,                      # a hair more: 70
        3000 ** 2 + 3000 ** 2 + 280000 ** 2: 1310,   # NEMO tower's longest pair
        3000 ** 2 + 3000 ** 2 + 520000 ** 2: 2414,   # KM3Net-It tower's longest pair
        633000 ** 2 + 273000 ** 2 + 520000 ** 2: 3995,  # array corner to corner
    }
    for d2, want in cases.items():
        assert oracle.dtmax_pair(d2) == want, d2
        assert 20 + _k_exact(d2) == want


def test_dtmax_tables_match_geometry(params):
    for make, want_max in ((workload.nemo_tower, 1310), (workload.km3_tower, 2414)):
        det = make()
        dt = oracle.dtmax(det.xyz_mm, params)
        assert dt.max() == want_max
        assert np.array_equal(dt, dt.T)
        assert np.all(np.diag(dt) == 20)


def test_dtmax_random_against_bigint_and_longdouble(params):
    rng = np.random.Generator(np.random.PCG64(7))
    xyz = rng.integers(-600_000, 600_000, size=(700, 3)).astype(np.int32)
    xyz[:50, 2] = 0
    xyz[50:100] = xyz[0]          # co-located PMTs
    dt = oracle.dtmax(xyz, params).astype(np.int64)
    d = xyz[:, None, :].astype(np.int64) - xyz[None, :, :].astype(np.int64)
    d2 = (d * d).sum(-1)
    # extended precision ceil, skipping values within 1e-9 of an integer
    x = np.sqrt(d2.astype(np.longdouble)) * np.longdouble(6900) / np.longdouble(1499000)
    c = np.ceil(x)
    ok = np.abs(x - np.round(x)) > 1e-9
    assert np.array_equal(dt[ok], 20 + c[ok].astype(np.int64))
    # the rest (and a sample of all) against the big-integer root
    idx = np.argwhere(~ok).tolist() + rng.integers(0, 700, size=(2000, 2)).tolist()
    for i, j in idx:
        assert dt[i, j] == 20 + _k_exact(int(d2[i, j])), (i, j)


# ------------------------------------------------------ all-pairs brute force

def _brute(det, par, hits, t0s):
    """Plain definition over every pair, no ordering and no window."""
    P = det.n_pmt
    xyz = det.xyz_mm.astype(np.int64)
    floor = det.floor_id
    W = par["corr_window_ns"]

    def dtm(a, b):
        dd = xyz[a] - xyz[b]
        return par["tol_ns"] + _k_exact(int((dd * dd).sum()), par["n_num"], par["n_den"])

    cache = {}
    H = [(int(h["t"]), int(h["pmt"]), int(h["charge"])) for h in hits]
    out = []
    for t0 in t0s:
        seeds = []
        for (ts, ps, qs) in H:
            if not (t0 <= ts < t0 + par["slice_ns"]):
                continue
            seed = qs >= par["q_seed_adc"]
            if not seed:
                seed = any(pj != ps and floor[pj] == floor[ps] and abs(tj - ts) <= par["floor_tau_ns"]
                           for (tj, pj, qj) in H)
            if not seed:
                continue
            c = 0
            for (tj, pj, qj) in H:
                key = (ps, pj)
                if key not in cache:
                    cache[key] = dtm(ps, pj)
                if abs(tj - ts) <= min(cache[key], W):
                    c += 1
            seeds.append((ts, ps, qs, c))
        seeds.sort()
        trig = [s for s in seeds if s[3] >= par["threshold"]]
        wins = []
        h = par["win_half_ns"]
        for s in sorted(trig):
            lo, hi = s[0] - h, s[0] + h
            if wins and lo <= wins[-1][1] + 1:
                wins[-1][1] = max(wins[-1][1], hi)
                wins[-1][3] += 1
            else:
                wins.append([lo, hi, 0, 1])
        for w in wins:
            w[2] = sum(1 for (tj, _, _) in H if w[0] <= tj <= w[1])
        out.append((seeds, trig, [tuple(w) for w in wins]))
    return out


@pytest.mark.parametrize("case", range(6))
def test_oracle_matches_all_pairs_bruteforce(case, params):
    rng = np.random.Generator(np.random.PCG64(100 + case))
    det = [workload.nemo_tower, workload.km3_tower][case % 2]()
    par = dict(params)
    par["slice_ns"] = 20_000
    par["threshold"] = int(rng.integers(1, 6))
    par["q_seed_adc"] = int(rng.choice([300, 150, 65535]))
    if case == 5:
        par["corr_window_ns"] = 400          # make the clamp bind on a tower
        par["win_half_ns"] = 500
    n = int(rng.integers(150, 320))
    t0s = [1_000_000, 1_020_000]
    t = rng.integers(1_000_000 - 3000, 1_040_000 + 3000, n)
    # forced near-coincidences and exact ties
    t[: n // 4] = t[n // 4: 2 * (n // 4)] + rng.integers(-25, 26, n // 4)
    t[-10:] = t[-20:-10]
    hits = np.zeros(n, oracle.HIT_DTYPE)
    hits["t"] = t
    hits["pmt"] = rng.integers(0, det.n_pmt, n)
    hits["charge"] = rng.integers(1, 400, n)
    got = oracle.run(det.xyz_mm, det.floor_id, par, hits, t0s)
    want = _brute(det, par, hits, t0s)
    for r, (seeds, trig, wins) in zip(got, want):
        assert _tuples(r.seeds, SEED_F) == seeds
        assert _tuples(r.triggers, SEED_F) == trig
        assert _tuples(r.windows, WIN_F) == wins


def test_merge_is_lexicographic_sort():
    rng = np.random.Generator(np.random.PCG64(3))
    h = np.zeros(5000, oracle.HIT_DTYPE)
    h["t"] = rng.integers(0, 300, 5000)
    h["pmt"] = rng.integers(0, 8, 5000)
    h["charge"] = rng.integers(0, 4, 5000)
    h["reserved"] = np.arange(5000)
    m = oracle.merge(h)
    order = np.lexsort((h["reserved"], h["charge"], h["pmt"], h["t"]))
    assert np.array_equal(m, h[order])


# ------------------------------------------------------------ closed forms

def test_accidental_floor_coincidence_rate(params):
    """Pure Poisson background, no charge seeds: a hit is a seed iff one of
    the other PMTs of its floor has a hit within +-tau.  For rates R_b the
    chance is 1 - exp(-sum_b R_b (2 tau + 1 ns)) (integer-ns times), the
    paper's 2 R^2 tau accidental rate per PMT pair at first order."""
    det = workload.nemo_tower()
    par = dict(params)
    par["q_seed_adc"] = 65535
    n_slices, rate = 50, 50e3
    S = par["slice_ns"]
    t_org = workload.T_ORIGIN_NS
    st = workload.gen_stream(det, t_org - 3000, t_org + n_slices * S + 3000, rate, seed=11, stream=77)
    t0s = [t_org + k * S for k in range(n_slices)]
    res = oracle.run(det.xyz_mm, det.floor_id, par, st.hits, t0s)
    obs = sum(len(r.seeds) for r in res)
    tau = par["floor_tau_ns"]
    lam = 3 * rate * (2 * tau + 1) * 1e-9           # three floor mates per PMT on NEMO
    n_hits = int(np.count_nonzero((st.hits["t"] >= t0s[0]) & (st.hits["t"] < t0s[-1] + S)))
    expect = n_hits * (1 - math.exp(-lam))
    sigma = math.sqrt(2 * expect)                    # seeds come in pairs
    assert abs(obs - expect) < 4 * sigma, (obs, expect, sigma)
    # without the +1 ns of integer time the expectation moves by > 4 sigma
    wrong = n_hits * (1 - math.exp(-3 * rate * 2 * tau * 1e-9))
    assert abs(wrong - expect) > 4 * sigma


def test_mean_causal_count_closed_form(params):
    """Every hit a seed (q_seed = 0), threshold 0: on Poisson background
    E[c(s) - 1] = sum_j R_j (2 min(dt_max[p_s][j], W) + 1 ns)."""
    det = workload.tower_array(nx=8, ny=2)            # 16 towers: 1344 PMTs, far pairs beyond 3 us
    par = dict(params)
    par.update(q_seed_adc=0, threshold=0, slice_ns=200_000)
    rate = 55e3
    n_slices = 150
    t_org = workload.T_ORIGIN_NS
    S = par["slice_ns"]
    st = workload.gen_stream(det, t_org - 3000, t_org + n_slices * S + 3000, rate, seed=5, stream=9)
    t0s = [t_org + k * S for k in range(n_slices)]
    res = oracle.run(det.xyz_mm, det.floor_id, par, st.hits, t0s)
    dt = np.minimum(oracle.dtmax(det.xyz_mm, par).astype(np.float64), par["corr_window_ns"])
    per_pmt = (rate * (2 * dt + 1) * 1e-9).sum(1)    # expected c-1 for a seed on PMT p
    means, expects = [], []
    for r in res:
        c = r.seeds["count"].astype(np.float64) - 1
        means.append(c.mean())
        expects.append(per_pmt[r.seeds["pmt"]].mean())
    means, expects = np.array(means), np.array(expects)
    err = means.std(ddof=1) / math.sqrt(len(means))
    assert abs(means.mean() - expects.mean()) < 4 * err + 1e-9, (means.mean(), expects.mean(), err)
    # a count that left out the seed itself would sit 1 lower: resolved
    assert abs(means.mean() + 1 - expects.mean()) > 4 * err, err


# ------------------------------------------------------ injection recovery

@pytest.mark.parametrize("cfg", ["nemo", "km3"])
def test_injected_tracks_above_threshold_are_recovered(cfg, params):
    wl = workload.CONFIGS[cfg]()
    det = wl.detectors[0]
    full = wl.runs[0]
    t0s = wl.run_slices[0]
    res = oracle.run(det.xyz_mm, det.floor_id, params, full.hits, t0s)
    trig = {}
    for r in res:
        for x in r.triggers:
            trig[(int(x["t"]), int(x["pmt"]), int(x["charge"]))] = int(x["count"])
    wins = np.concatenate([r.windows for r in res])
    tracks = np.unique(full.hits["reserved"][full.hits["reserved"] > 0])
    n_above = 0
    for m in tracks:
        own = full.hits[full.hits["reserved"] == m]
        alone = oracle.run(det.xyz_mm, det.floor_id, params, own, t0s)
        for r in alone:
            for x in r.triggers:
                n_above += 1
                key = (int(x["t"]), int(x["pmt"]), int(x["charge"]))
                assert key in trig, (m, key)
                assert trig[key] >= int(x["count"])
                inside = (wins["lo"] <= x["t"] - params["win_half_ns"]) & (wins["hi"] >= x["t"] + params["win_half_ns"])
                assert inside.any()
    assert n_above > 0


# ------------------------------------------------------------- invariance

def test_trigger_list_independent_of_slicing(params):
    wl = workload.cfg_km3()
    det = wl.detectors[0]
    full = wl.runs[0]
    a = oracle.run(det.xyz_mm, det.floor_id, params, full.hits, wl.run_slices[0])
    par2 = dict(params)
    par2["slice_ns"] = params["slice_ns"] // 4
    t0 = wl.run_slices[0][0]
    b = oracle.run(det.xyz_mm, det.floor_id, par2, full.hits,
                   [t0 + k * par2["slice_ns"] for k in range(4 * len(wl.run_slices[0]))])
    ta = np.concatenate([r.triggers for r in a])
    tb = np.concatenate([r.triggers for r in b])
    sa = np.concatenate([r.seeds for r in a])
    sb = np.concatenate([r.seeds for r in b])
    assert np.array_equal(ta, tb)
    assert np.array_equal(sa, sb)
    # shuffling the input does not change anything
    perm = np.random.Generator(np.random.PCG64(1)).permutation(len(full.hits))
    c = oracle.run(det.xyz_mm, det.floor_id, params, full.hits[perm], wl.run_slices[0])
    for x, y in zip(a, c):
        assert np.array_equal(x.triggers, y.triggers)
        assert np.array_equal(x.windows, y.windows)


# ------------------------------------------------------------ event payload

def test_events_golden_fixture():
    """The windows fixture's event payload, derived by hand: window 1 holds
    the seeds at 400000 and 406001 and the PMT 1 hit at its inclusive end
    409001; the PMT 1 hit at 409002 is in the gap; window 2 holds 409003 (its
    inclusive start) and the seed at 412003; window 3 the two PMT 20 seeds."""
    fx = json.load(open(os.path.join(GOLDEN, "windows_nemo32.json")))
    g = workload.nemo_tower()
    par = dict(workload.DEFAULT_PARAMS, **fx["params"])
    hits = np.zeros(len(fx["hits"]), oracle.HIT_DTYPE)
    for i, (t, p, q) in enumerate(fx["hits"]):
        hits[i] = (t, p, q, 0)
    res = oracle.run(g.xyz_mm, g.floor_id, par, hits, fx["slices"])[0]
    ev = oracle.events(hits, res.windows)
    expect = [1000400000, 1000406001, 1000409001, 1000409003, 1000412003, 1000500000, 1000506000]
    assert ev["t"].tolist() == expect
    assert len(ev) == int(res.windows["n_hits"].sum())


def test_events_bruteforce_and_window_counts():
    """On random dense slices: the payload equals a plain double loop over
    windows and hits, and its size equals the windows' hit counts that the
    C oracle computes independently."""
    rng = np.random.Generator(np.random.PCG64(77))
    g = workload.nemo_tower()
    for case in range(6):
        par = dict(workload.DEFAULT_PARAMS, slice_ns=50_000, threshold=int(rng.integers(1, 5)),
                   win_half_ns=int(rng.integers(50, 3000)))
        t0 = 10_000_000
        n = int(rng.integers(50, 400))
        hits = np.zeros(n, oracle.HIT_DTYPE)
        hits["t"] = rng.integers(t0 - 3000, t0 + par["slice_ns"] + 3000, n)
        hits["pmt"] = rng.integers(0, 32, n)
        hits["charge"] = rng.integers(1, 500, n)
        res = oracle.run(g.xyz_mm, g.floor_id, par, hits, [t0])[0]
        ev = oracle.events(hits, res.windows)
        want = []
        for h in sorted(hits.tolist(), key=lambda x: (x[0], x[1], x[2])):
            if any(lo <= h[0] <= hi for lo, hi, _, _ in res.windows.tolist()):
                want.append(h[:3])
        assert [tuple(x)[:3] for x in ev.tolist()] == [tuple(x) for x in want], case
        assert len(ev) == int(res.windows["n_hits"].sum()), case


# ------------------------------------------------------------------ level 0

def _fixture_hits(fx):
    hits = np.zeros(len(fx["hits"]), oracle.HIT_DTYPE)
    for i, (t, p, q) in enumerate(fx["hits"]):
        hits[i] = (t, p, q, 0)
    return hits


def test_level0_golden_fixture():
    fx = json.load(open(os.path.join(GOLDEN, "level0", "nemo32.json")))
    g = workload.nemo_tower()
    hits = _fixture_hits(fx)
    base = dict(workload.DEFAULT_PARAMS, **fx["params"])
    for mode, par in (("off", dict(base, l0_hits=0)), ("count", base), ("distinct", dict(base, l0_distinct_pmts=1))):
        res = oracle.run(g.xyz_mm, g.floor_id, par, hits, fx["slices"])[0]
        assert res.seeds["t"].tolist() == fx["expected_seed_times"][mode], mode


def _level0_brute(sorted_hits, s, n_req, tw, distinct):
    """Level 0 at sorted hit s by every window start a in (t_s - TW, t_s]."""
    t = sorted_hits["t"]
    ts = int(t[s])
    for a in sorted(set(int(x) for x in t if ts - tw < x <= ts)):
        inside = sorted_hits[(t >= a) & (t < a + tw)]
        k = len(set(inside["pmt"].tolist())) if distinct else len(inside)
        if k >= n_req:
            return True
    return False


def test_level0_bruteforce_and_index_reading():
    """Random dense slices: the oracle's level-0 keeps exactly the seeds a
    direct window search keeps, with unchanged counts; for the hit count the
    paper's index form t[i + N - 1] - t[i] < TW over consecutive merged
    hits keeps the same seeds."""
    rng = np.random.Generator(np.random.PCG64(123))
    g = workload.nemo_tower()
    for case in range(8):
        n_req = int(rng.integers(2, 8))
        tw = int(rng.choice([50, 200, 1000]))
        distinct = int(case % 2)
        par = dict(workload.DEFAULT_PARAMS, slice_ns=40_000, threshold=1, l0_window_ns=tw,
                   l0_distinct_pmts=distinct, q_seed_adc=250)
        t0 = 10_000_000
        n = int(rng.integers(100, 500))
        hits = np.zeros(n, oracle.HIT_DTYPE)
        hits["t"] = rng.integers(t0 - 3000, t0 + par["slice_ns"] + 3000, n)
        hits["pmt"] = rng.integers(0, 32, n)
        hits["charge"] = rng.integers(1, 400, n)
        off = oracle.run(g.xyz_mm, g.floor_id, dict(par, l0_hits=0), hits, [t0])[0]
        on = oracle.run(g.xyz_mm, g.floor_id, dict(par, l0_hits=n_req), hits, [t0])[0]
        sh = oracle.merge(hits)
        key = list(zip(sh["t"].tolist(), sh["pmt"].tolist(), sh["charge"].tolist()))
        keep = []
        for sd in off.seeds.tolist():
            s = key.index(tuple(sd[:3]))
            if _level0_brute(sh, s, n_req, tw, distinct):
                keep.append(sd)
        assert on.seeds.tolist() == keep, case
        if not distinct:
            idx = []
            for sd in off.seeds.tolist():
                s = key.index(tuple(sd[:3]))
                ok = any(0 <= i and i + n_req - 1 < len(sh) and int(sh["t"][i + n_req - 1]) - int(sh["t"][i]) < tw
                         for i in range(s - n_req + 1, s + 1))
                if ok:
                    idx.append(sd)
            assert idx == keep, case


def test_distinct_level0_bruteforce_above_128_pmts():
    """The distinct-PMT level 0 on a 168-PMT two-tower array (PMT ids above
    128, repeats of one PMT inside a window): the oracle keeps exactly the
    seeds whose some window holds N different PMTs."""
    rng = np.random.Generator(np.random.PCG64(321))
    g = workload.tower_array(nx=2, ny=1)
    for case in range(6):
        n_req = int(rng.integers(2, 9))
        tw = int(rng.choice([100, 400, 1000]))
        par = dict(workload.DEFAULT_PARAMS, slice_ns=30_000, threshold=1, l0_window_ns=tw, l0_hits=n_req,
                   l0_distinct_pmts=1, q_seed_adc=250)
        t0 = 10_000_000
        n = int(rng.integers(150, 400))
        hits = np.zeros(n, oracle.HIT_DTYPE)
        hits["t"] = rng.integers(t0 - 3000, t0 + par["slice_ns"] + 3000, n)
        hits["pmt"] = rng.choice(np.r_[rng.integers(0, 168, 12), rng.integers(128, 168, 6)], n)
        hits["charge"] = rng.integers(1, 400, n)
        off = oracle.run(g.xyz_mm, g.floor_id, dict(par, l0_hits=0), hits, [t0])[0]
        on = oracle.run(g.xyz_mm, g.floor_id, par, hits, [t0])[0]
        sh = oracle.merge(hits)
        key = list(zip(sh["t"].tolist(), sh["pmt"].tolist(), sh["charge"].tolist()))
        keep = [sd for sd in off.seeds.tolist() if _level0_brute(sh, key.index(tuple(sd[:3])), n_req, tw, 1)]
        assert on.seeds.tolist() == keep, case
        assert 0 < len(keep) <= len(off.seeds), case


# ------------------------------------- coincidence ladder, distinct count

def test_ladder_golden_fixture():
    fx = json.load(open(os.path.join(GOLDEN, "ladder", "nemo32.json")))
    g = workload.nemo_tower()
    hits = _fixture_hits(fx)
    for name, v in fx["variants"].items():
        par = dict(workload.DEFAULT_PARAMS, **fx["params"])
        par.update(v["params"])
        res = oracle.run(g.xyz_mm, g.floor_id, par, hits, fx["slices"])[0]
        assert res.seeds["t"].tolist() == v["seed_times"], name
        assert res.triggers["t"].tolist() == v["seed_times"], name      # threshold 1: every seed fires


def test_distinct_count_golden_fixture():
    fx = json.load(open(os.path.join(GOLDEN, "distinct", "nemo32.json")))
    g = workload.nemo_tower()
    hits = _fixture_hits(fx)
    for mode, flag in (("count", 0), ("distinct", 1)):
        par = dict(workload.DEFAULT_PARAMS, **fx["params"], count_distinct_pmts=flag)
        res = oracle.run(g.xyz_mm, g.floor_id, par, hits, fx["slices"])[0]
        assert _tuples(res.seeds, SEED_F) == [tuple(x) for x in fx["expected_seeds"][mode]], mode


def _floor_levels(det):
    """Per PMT: position of its floor among its tower's floors, ordered by
    the height of each floor's lowest PMT, then floor id (pure Python)."""
    lowest = {}
    for p in range(det.n_pmt):
        f = int(det.floor_id[p])
        lowest[f] = min(lowest.get(f, 1 << 62), int(det.xyz_mm[p][2]))
    order = {}
    for p in range(det.n_pmt):
        order.setdefault(int(det.tower_id[p]), set()).add((lowest[int(det.floor_id[p])], int(det.floor_id[p])))
    pos = {tw: {f: i for i, (_, f) in enumerate(sorted(s))} for tw, s in order.items()}
    return [pos[int(det.tower_id[p])][int(det.floor_id[p])] for p in range(det.n_pmt)]


def _brute_ext(det, par, hits, t0):
    """All pairs, no ordering: the coincidence ladder (seed rule 1) with its
    level-0 filter off, and the causal count of hits or of different PMTs."""
    xyz = [tuple(int(c) for c in row) for row in det.xyz_mm]
    floor = [int(f) for f in det.floor_id]
    tower = [int(x) for x in det.tower_id]
    level = _floor_levels(det)
    W = par["corr_window_ns"]
    H = [(int(h["t"]), int(h["pmt"]), int(h["charge"])) for h in hits]

    def d2(a, b):
        return sum((xyz[a][c] - xyz[b][c]) ** 2 for c in range(3))

    def is_seed(i):
        ts, ps, qs = H[i]
        if par["seed_rule"] == 0:
            return qs >= par["q_seed_adc"] or any(
                pj != ps and floor[pj] == floor[ps] and abs(tj - ts) <= par["floor_tau_ns"] for (tj, pj, _) in H)
        sc = fc = afc = False
        for j, (tj, pj, _) in enumerate(H):
            if j == i:
                continue
            d = abs(tj - ts)
            same_floor = pj != ps and floor[pj] == floor[ps]
            sc |= same_floor and d2(ps, pj) <= par["sc_dist_mm"] ** 2 and d <= par["sc_window_ns"]
            fc |= same_floor and d <= par["fc_window_ns"]
            afc |= tower[pj] == tower[ps] and abs(level[pj] - level[ps]) == 1 and d <= par["afc_window_ns"]
        return (sc and afc) or (fc and afc)

    out = []
    for i, (ts, ps, qs) in enumerate(H):
        if not (t0 <= ts < t0 + par["slice_ns"]) or not is_seed(i):
            continue
        rel = [pj for (tj, pj, _) in H if abs(tj - ts) <= min(par["tol_ns"] + _k_exact(d2(ps, pj), par["n_num"],
                                                                                      par["n_den"]), W)]
        c = len(set(rel)) if par["count_distinct_pmts"] else len(rel)
        out.append((ts, ps, qs, c))
    return sorted(out)


def _ladder_clusters(rng, det, lo, hi):
    """Random hits plus clusters of 3-8 hits within a few hundred ns on one
    floor, its neighbours in height (any tower) and the same PMT (ties and
    repeats included), so that every coincidence type occurs."""
    by_z = {}
    for p in range(det.n_pmt):
        by_z.setdefault(int(det.xyz_mm[p][2]), []).append(p)
    zs = sorted(by_z)
    rows = [(int(x), int(rng.integers(0, det.n_pmt)), int(rng.integers(1, 400)))
            for x in rng.integers(lo, hi, 60)]
    for _ in range(int(rng.integers(25, 40))):
        c = int(rng.integers(lo, hi))
        k = int(rng.integers(0, len(zs)))
        pool = by_z[zs[k]] + (by_z[zs[k - 1]] if k else []) + (by_z[zs[k + 1]] if k + 1 < len(zs) else [])
        if rng.random() < 0.7:          # mostly one tower
            tw = det.tower_id[pool[int(rng.integers(0, len(pool)))]]
            pool = [p for p in pool if det.tower_id[p] == tw]
        for _ in range(int(rng.integers(3, 9))):
            rows.append((c + int(rng.integers(-150, 151)), int(rng.choice(pool)), int(rng.integers(1, 400))))
    rows += rows[-3:]
    hits = np.zeros(len(rows), oracle.HIT_DTYPE)
    for i, (t, p, q) in enumerate(rows):
        hits[i] = (t, p, q, 0)
    return hits


@pytest.mark.parametrize("case", range(8))
def test_ladder_and_distinct_count_match_bruteforce(case, params):
    """Tiny dense slices on a tower and on a two-tower array (tower ids
    matter for AFC): the oracle's seeds and counts equal the all-pairs
    definition for both seed rules and both count forms."""
    rng = np.random.Generator(np.random.PCG64(700 + case))
    det = [workload.nemo_tower, workload.km3_tower, lambda: workload.tower_array(nx=2, ny=1)][case % 3]()
    par = dict(params, slice_ns=10_000, threshold=1, seed_rule=int(case % 2 == 0),
               count_distinct_pmts=int(case % 4 < 2),
               sc_window_ns=int(rng.choice([20, 60])), fc_window_ns=int(rng.choice([10, 100])),
               afc_window_ns=int(rng.choice([100, 250])), sc_dist_mm=int(rng.choice([1000, 7000])))
    t0 = 2_000_000
    hits = _ladder_clusters(rng, det, t0 - 3000, t0 + par["slice_ns"] + 3000)
    got = oracle.run(det.xyz_mm, det.floor_id, par, hits, [t0], tower_id=det.tower_id)[0]
    want = _brute_ext(det, par, hits, t0)
    assert len(want) >= 10, case
    assert _tuples(got.seeds, SEED_F) == want, case


def test_oracle_pmt_limit(params):
    """The oracle takes detectors of 1 to 4096 PMTs (its distinct-PMT forms
    keep a 4096-entry mark array per seed) and refuses larger ones instead
    of overrunning that array.  At the limit, the distinct count of seeds
    with hits on PMT 4095 equals the all-pairs definition."""
    from types import SimpleNamespace
    rng = np.random.Generator(np.random.PCG64(41))
    P = 4096
    xyz = np.zeros((P, 3), np.int32)
    xyz[:, 0] = rng.integers(-3000, 3000, P)                  # a 6 m cube: every pair causal within ~48 ns
    xyz[:, 1] = rng.integers(-3000, 3000, P)
    xyz[:, 2] = rng.integers(-3000, 3000, P)
    det = SimpleNamespace(n_pmt=P, xyz_mm=xyz, floor_id=np.arange(P, dtype=np.uint32) // 4,
                          tower_id=np.zeros(P, np.uint32))
    t0 = 1_000_000
    pm = [4095, 4094, 4095, 4093, 4092, 0, 1, 4095, 4095, 2]
    hits = np.zeros(len(pm), oracle.HIT_DTYPE)
    hits["t"] = t0 + 100 + 7 * np.arange(len(pm))
    hits["pmt"] = pm
    hits["charge"] = 400                                        # every hit is a charge seed
    par = dict(params, slice_ns=10_000, threshold=1, count_distinct_pmts=1)
    got = oracle.run(det.xyz_mm, det.floor_id, par, hits, [t0], tower_id=det.tower_id)[0]
    want = _brute_ext(det, par, hits, t0)
    assert _tuples(got.seeds, SEED_F) == want
    assert max(c for (_, _, _, c) in want) >= 5                 # repeats of PMT 4095 counted once
    for bad in (0, P + 1):
        with pytest.raises(RuntimeError):
            oracle.run(np.zeros((bad, 3), np.int32), np.zeros(bad, np.uint32), par, hits[:0], [t0])


def test_ladder_accidental_rate_closed_form(params):
    """Pure Poisson background, the paper's windows: a hit on PMT p is a
    seed iff another PMT of its floor has a hit within +-fc (SC implies FC
    here: adjacent PMTs share the floor and sc <= fc) and a PMT of a
    consecutive floor one within +-afc.  The two sets of PMTs are disjoint,
    so P = (1 - exp(-lam_fc)) (1 - exp(-lam_afc)), lam = sum R (2 w + 1 ns).
    The top and bottom floors have one consecutive floor, the others two."""
    det = workload.nemo_tower()
    par = dict(params, seed_rule=1, threshold=1)
    n_slices, rate = 40, 50e3
    S = par["slice_ns"]
    t_org = workload.T_ORIGIN_NS
    st = workload.gen_stream(det, t_org - 3000, t_org + n_slices * S + 3000, rate, seed=21, stream=81)
    t0s = [t_org + k * S for k in range(n_slices)]
    res = oracle.run(det.xyz_mm, det.floor_id, par, st.hits, t0s)
    obs = sum(len(r.seeds) for r in res)
    own = st.hits[(st.hits["t"] >= t0s[0]) & (st.hits["t"] < t0s[-1] + S)]
    n_floors = int(det.floor_id.max()) + 1
    fl = det.floor_id[own["pmt"]]
    n_next = np.where((fl == 0) | (fl == n_floors - 1), 4, 8)
    lam_fc = 3 * rate * (2 * par["fc_window_ns"] + 1) * 1e-9
    lam_afc = n_next * rate * (2 * par["afc_window_ns"] + 1) * 1e-9
    expect = float(((1 - math.exp(-lam_fc)) * (1 - np.exp(-lam_afc))).sum())
    sigma = math.sqrt(3 * expect)
    assert abs(obs - expect) < 4 * sigma, (obs, expect, sigma)
    # counting a single consecutive floor everywhere moves it by far more
    wrong = float(((1 - math.exp(-lam_fc)) * (1 - np.exp(-4 * rate * (2 * par["afc_window_ns"] + 1) * 1e-9))).sum())
    assert abs(wrong - expect) > 4 * sigma


def test_distinct_count_closed_form(params):
    """Every hit a seed, distinct-PMT count, Poisson background on the
    84-PMT tower at a high rate: E[c(s) - 1] = sum_{q != p_s} (1 -
    exp(-R (2 min(dt_max[p_s][q], W) + 1 ns))) -- the seed's own PMT is
    always in the set; every other PMT is in it iff it has a hit in its
    range.  The plain count's expectation sum R (2 dt + 1) is far off."""
    det = workload.km3_tower()
    par = dict(params, q_seed_adc=0, threshold=0, slice_ns=100_000, count_distinct_pmts=1)
    rate = 400e3
    n_slices = 40
    t_org = workload.T_ORIGIN_NS
    S = par["slice_ns"]
    st = workload.gen_stream(det, t_org - 3000, t_org + n_slices * S + 3000, rate, seed=31, stream=91)
    t0s = [t_org + k * S for k in range(n_slices)]
    res = oracle.run(det.xyz_mm, det.floor_id, par, st.hits, t0s)
    dt = np.minimum(oracle.dtmax(det.xyz_mm, par).astype(np.float64), par["corr_window_ns"])
    lam = rate * (2 * dt + 1) * 1e-9
    np.fill_diagonal(lam, 0.0)
    per_pmt = (1 - np.exp(-lam)).sum(1)
    per_pmt_plain = lam.sum(1)
    means, expects, plains = [], [], []
    for r in res:
        means.append(r.seeds["count"].astype(np.float64).mean() - 1)
        expects.append(per_pmt[r.seeds["pmt"]].mean())
        plains.append(per_pmt_plain[r.seeds["pmt"]].mean())
    means = np.array(means)
    err = means.std(ddof=1) / math.sqrt(len(means))
    assert abs(means.mean() - np.mean(expects)) < 4 * err + 1e-9, (means.mean(), np.mean(expects), err)
    assert abs(means.mean() - np.mean(plains)) > 4 * err


# ------------------------------------------------------ multi-tower selection

def _array_case(fx_hits_rel, t0, tower_par):
    g = workload.tower_array(nx=2, ny=1)
    towers = workload.split_towers(g)
    streams = [workload.stream_from_rows([(t0 + t, p, q) for (t, p, q) in rows], 84) for rows in fx_hits_rel]
    seeds = [oracle.run(tw.xyz_mm, tw.floor_id, tower_par, st.hits, [t0])[0].triggers for tw, st in zip(towers, streams)]
    return towers, streams, seeds


def test_array_selection_golden_fixture():
    import oracle.array as oa
    fx = json.load(open(os.path.join(GOLDEN, "array", "two_towers.json")))
    t0 = fx["t0"]
    tower_par = dict(workload.DEFAULT_PARAMS, **fx["tower_params"])
    towers, streams, seeds = _array_case(fx["hits_rel"], t0, tower_par)
    for name, v in fx["variants"].items():
        ap = dict(fx["array_params"], **v["array_params"])
        r = oa.select([tw.xyz_mm for tw in towers], tower_par, ap["min_towers"], ap["corr_window_ns"],
                      ap["win_half_ns"], seeds, [(st.hits, st.pmt_off) for st in streams])
        assert [[int(s["t"]) - t0, int(s["pmt"]), int(s["tower"]), int(s["n_towers"])] for s in r.seeds] == \
            v["seeds_rel"], name
        assert [[int(w["lo"]) - t0, int(w["hi"]) - t0, int(w["n_hits"]), int(w["n_triggers"])] for w in r.windows] \
            == v["windows_rel"], name
        frags = [[[int(h["t"]) - t0, int(h["pmt"]), int(h["charge"])] for h in r.hits[int(a):int(b)]]
                 for a, b in zip(r.frag_off[:-1], r.frag_off[1:])]
        assert frags == v["fragments_rel"], name


def _array_brute(tower_xyz, par, K, W, h, seeds, streams):
    """All pairs of seeds, the distance in pure Python, no search."""
    allp = [(b, s) for b, S in enumerate(seeds) for s in S.tolist()]
    out = []
    for a, s in allp:
        ts, ps = s[0], s[1]
        tw = set()
        for b, j in allp:
            d = sum((int(tower_xyz[a][ps][c]) - int(tower_xyz[b][j[1]][c])) ** 2 for c in range(3))
            lim = min(par["tol_ns"] + _k_exact(d, par["n_num"], par["n_den"]), W)
            if abs(j[0] - ts) <= lim:
                tw.add(b)
        if len(tw) >= K:
            out.append((ts, a, s, len(tw)))
    out.sort(key=lambda x: (x[0], x[1]))
    sel = [(x[0], x[2][1], x[1], x[3]) for x in out]
    wins = []
    for (t, _, _, _) in sel:
        if wins and t - h <= wins[-1][1] + 1:
            wins[-1][1] = max(wins[-1][1], t + h)
            wins[-1][2] += 1
        else:
            wins.append([t - h, t + h, 1])
    frags = []
    for lo, hi, _ in wins:
        for b, (hits, off) in enumerate(streams):
            frags.append([(int(x["t"]), int(x["pmt"]), int(x["charge"])) for x in hits if lo <= int(x["t"]) <= hi])
    return sel, [(lo, hi, k) for lo, hi, k in wins], frags


@pytest.mark.parametrize("case", range(4))
def test_array_selection_matches_bruteforce(case, params):
    """Random seeds on two or three towers: selection, windows and readback
    equal the all-pairs definition."""
    import oracle.array as oa
    rng = np.random.Generator(np.random.PCG64(1300 + case))
    g = workload.tower_array(nx=2 + case % 2, ny=1)
    towers = workload.split_towers(g)
    par = dict(params, threshold=1, slice_ns=40_000)
    t0 = 3_000_000
    K = int(rng.integers(1, 4))
    W, h = int(rng.choice([600, 3000])), int(rng.choice([500, 3000]))
    streams, seeds = [], []
    centers = rng.integers(t0, t0 + par["slice_ns"], 12)
    for tw in towers:
        rows = []
        for c in centers:
            for _ in range(int(rng.integers(0, 3))):
                rows.append((int(c + rng.integers(-700, 701)), int(rng.integers(0, 84)), 300))
        for _ in range(30):
            rows.append((int(rng.integers(t0 - 4000, t0 + par["slice_ns"] + 4000)), int(rng.integers(0, 84)),
                         int(rng.integers(1, 300))))
        st = workload.stream_from_rows(rows, 84)
        streams.append(st)
        seeds.append(oracle.run(tw.xyz_mm, tw.floor_id, par, st.hits, [t0])[0].triggers)
    r = oa.select([tw.xyz_mm for tw in towers], par, K, W, h, seeds, [(s.hits, s.pmt_off) for s in streams])
    sel, wins, frags = _array_brute([tw.xyz_mm for tw in towers], par, K, W, h, seeds,
                                    [(s.hits, s.pmt_off) for s in streams])
    assert len(sel) > 0
    assert [(int(s["t"]), int(s["pmt"]), int(s["tower"]), int(s["n_towers"])) for s in r.seeds] == sel
    assert [(int(w["lo"]), int(w["hi"]), int(w["n_triggers"])) for w in r.windows] == wins
    got = [[(int(x["t"]), int(x["pmt"]), int(x["charge"])) for x in r.hits[int(a):int(b)]]
           for a, b in zip(r.frag_off[:-1], r.frag_off[1:])]
    assert got == frags
    assert [int(w["n_hits"]) for w in r.windows] == [
        sum(len(f) for f in frags[k * len(towers):(k + 1) * len(towers)]) for k in range(len(wins))]
