"""Seeded synthetic inputs for the muon-trigger workloads.

Shared by the CPU oracle's tests and by the GPU library's tests and
benchmarks.  It draws detectors (PMT positions, floors, towers), Poisson
background, straight muon tracks and bioluminescence bursts; it holds none
of the trigger's arithmetic.

Detector geometry follows the NEMO Phase II tower (8 floors at 40 m, a 6 m
bar per floor) and the 14-floor KM3Net-It tower described in the paper's
"DAQ system of NEMO Phase II" and "Results" sections, plus a 32-tower array
of KM3Net-It-style towers.  PMT placement within a floor, the rotation of
odd floors and the tower grid are readings of the paper's silent points and
are listed with the other readings in the design notes.

The paper's own simulated data is not available; these generators stand in
for it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HIT_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("charge", "<u2"), ("reserved", "<u4")])
assert HIT_DTYPE.itemsize == 16

SLICE_NS = 200_000_000          # 200 ms time slices (paper, "DAQ system")
HALO_NS = 3_000                 # 3 us correlation interval / +-3 us event window
T_ORIGIN_NS = 1_000_000_000     # run start; keeps halo times positive

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libtrig_gen.so")


def build(force: bool = False) -> str:
    """Compile gen.c into libtrig_gen.so (portable C, no arch flags)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


class _Spec(ctypes.Structure):
    _fields_ = [
        ("n_pmt", ctypes.c_uint32),
        ("xyz_mm", ctypes.POINTER(ctypes.c_int32)),
        ("t_begin_ns", ctypes.c_int64),
        ("t_end_ns", ctypes.c_int64),
        ("rate_hz", ctypes.POINTER(ctypes.c_double)),
        ("n_muons", ctypes.c_uint32),
        ("muon_margin_ns", ctypes.c_int64),
        ("muon_pe_scale", ctypes.c_double),
        ("muon_att_m", ctypes.c_double),
        ("muon_max_d_m", ctypes.c_double),
        ("muon_jitter_ns", ctypes.c_double),
        ("cherenkov_deg", ctypes.c_double),
        ("refr_index", ctypes.c_double),
        ("box_grow_m", ctypes.c_double),
        ("n_bursts", ctypes.c_uint32),
        ("burst_len_ns", ctypes.c_int64),
        ("burst_rate_hz", ctypes.c_double),
        ("burst_pmts", ctypes.c_uint32),
        ("pe_adc", ctypes.c_double),
        ("pe_sigma_adc", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_uint64),
        ("n_threads", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gen_stream.restype = ctypes.c_void_p
        lib.gen_stream.argtypes = [ctypes.POINTER(_Spec), ctypes.POINTER(ctypes.c_uint64)]
        lib.gen_stream_copy.restype = None
        lib.gen_stream_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.gen_stream_free.restype = None
        lib.gen_stream_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


# --------------------------------------------------------------- detectors

@dataclass
class Detector:
    """PMT positions (integer mm), floor ids (equal id = same floor) and tower ids."""
    name: str
    xyz_mm: np.ndarray      # (P, 3) int32
    floor_id: np.ndarray    # (P,) uint32
    tower_id: np.ndarray    # (P,) uint32

    @property
    def n_pmt(self) -> int:
        return int(self.xyz_mm.shape[0])


def _tower(n_floors: int, xs_m, x0_m=0.0, y0_m=0.0, floor_base=0, tower=0):
    """One tower: floors at z = 40 m * k; on each floor two co-located PMTs at
    every x in xs_m along the bar; odd floors are rotated by 90 degrees."""
    xyz, floors, towers = [], [], []
    for k in range(n_floors):
        for x in xs_m:
            for _ in range(2):
                if k % 2 == 0:
                    pos = (x0_m + x, y0_m, 40.0 * k)
                else:
                    pos = (x0_m, y0_m + x, 40.0 * k)
                xyz.append([round(c * 1000.0) for c in pos])
                floors.append(floor_base + k)
                towers.append(tower)
    return xyz, floors, towers


def nemo_tower() -> Detector:
    """NEMO Phase II: 8 floors, 40 m apart, 6 m bar, 2 PMTs at each end (32 PMTs)."""
    xyz, fl, tw = _tower(8, (-3.0, 3.0))
    return Detector("nemo32", np.asarray(xyz, np.int32), np.asarray(fl, np.uint32), np.asarray(tw, np.uint32))


def km3_tower() -> Detector:
    """KM3Net-It tower: 14 floors at 40 m, 6 PMTs per floor (84 PMTs)."""
    xyz, fl, tw = _tower(14, (-3.0, 0.0, 3.0))
    return Detector("km3it84", np.asarray(xyz, np.int32), np.asarray(fl, np.uint32), np.asarray(tw, np.uint32))


def tower_array(nx: int = 8, ny: int = 4, pitch_m: float = 90.0) -> Detector:
    """nx * ny KM3Net-It-style towers on a square grid (default 32 towers, 2688 PMTs)."""
    xyz, fl, tw = [], [], []
    for j in range(ny):
        for i in range(nx):
            t = j * nx + i
            a, b, c = _tower(14, (-3.0, 0.0, 3.0), x0_m=pitch_m * i, y0_m=pitch_m * j,
                             floor_base=14 * t, tower=t)
            xyz += a
            fl += b
            tw += c
    return Detector(f"array{nx * ny * 84}", np.asarray(xyz, np.int32), np.asarray(fl, np.uint32),
                    np.asarray(tw, np.uint32))


# ----------------------------------------------------------------- streams

@dataclass
class Stream:
    """Hits grouped by PMT (CSR): hits[pmt_off[p]:pmt_off[p+1]] is PMT p's
    time-ordered stream."""
    hits: np.ndarray        # HIT_DTYPE
    pmt_off: np.ndarray     # (P+1,) uint64

    @property
    def n_hits(self) -> int:
        return int(self.pmt_off[-1])


def gen_stream(det: Detector, t_begin: int, t_end: int, rate_hz, *, n_muons: int = 0,
               n_bursts: int = 0, burst_len_ns: int = 10_000_000, burst_rate_hz: float = 500e3,
               burst_pmts: int = 3, seed: int = 0, stream: int = 0, threads: int | None = None) -> Stream:
    lib = _load()
    P = det.n_pmt
    rates = np.broadcast_to(np.asarray(rate_hz, np.float64), (P,)).copy()
    xyz = np.ascontiguousarray(det.xyz_mm, np.int32).reshape(-1)
    sp = _Spec()
    sp.n_pmt = P
    sp.xyz_mm = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    sp.t_begin_ns = int(t_begin)
    sp.t_end_ns = int(t_end)
    sp.rate_hz = rates.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    sp.n_muons = n_muons
    sp.muon_margin_ns = 10_000
    sp.muon_pe_scale = 3.0
    sp.muon_att_m = 40.0
    sp.muon_max_d_m = 100.0
    sp.muon_jitter_ns = 3.0
    sp.cherenkov_deg = 41.0
    sp.refr_index = 1.38
    sp.box_grow_m = 100.0
    sp.n_bursts = n_bursts
    sp.burst_len_ns = burst_len_ns
    sp.burst_rate_hz = burst_rate_hz
    sp.burst_pmts = burst_pmts
    sp.pe_adc = 100.0
    sp.pe_sigma_adc = 40.0
    sp.seed = seed & 0xFFFFFFFFFFFFFFFF
    sp.stream = stream & 0xFFFFFFFFFFFFFFFF
    sp.n_threads = int(threads or os.cpu_count() or 1)
    n = ctypes.c_uint64(0)
    h = lib.gen_stream(ctypes.byref(sp), ctypes.byref(n))
    if not h:
        raise MemoryError("hit generator failed")
    try:
        hits = np.empty(n.value, HIT_DTYPE)
        off = np.empty(P + 1, np.uint64)
        lib.gen_stream_copy(h, hits.ctypes.data, off.ctypes.data)
    finally:
        lib.gen_stream_free(h)
    return Stream(hits, off)


def cut(stream: Stream, lo: int, hi: int) -> Stream:
    """Hits with lo <= t < hi, still grouped by PMT (a slice submission)."""
    off = stream.pmt_off.astype(np.int64)
    t = stream.hits["t"]
    P = len(off) - 1
    starts = np.empty(P, np.int64)
    ends = np.empty(P, np.int64)
    for p in range(P):
        a, b = off[p], off[p + 1]
        seg = t[a:b]
        starts[p] = a + np.searchsorted(seg, lo, "left")
        ends[p] = a + np.searchsorted(seg, hi, "left")
    lens = ends - starts
    new_off = np.zeros(P + 1, np.uint64)
    np.cumsum(lens, out=new_off[1:])
    total = int(new_off[-1])
    idx = np.repeat(starts - new_off[:-1].astype(np.int64), lens) + np.arange(total, dtype=np.int64)
    return Stream(stream.hits[idx], new_off)


def concat_streams(parts: list[Stream]) -> Stream:
    """Per-PMT concatenation of streams that follow each other in time."""
    P = len(parts[0].pmt_off) - 1
    segs, lens = [], np.zeros(P, np.int64)
    for p in range(P):
        for s in parts:
            a, b = int(s.pmt_off[p]), int(s.pmt_off[p + 1])
            segs.append(s.hits[a:b])
            lens[p] += b - a
    off = np.zeros(P + 1, np.uint64)
    np.cumsum(lens, out=off[1:])
    return Stream(np.concatenate(segs) if segs else np.empty(0, HIT_DTYPE), off)


def split_towers(det: Detector) -> list[Detector]:
    """The towers of an array as detectors of their own, PMTs renumbered
    from 0 in their array order, positions kept in the array's frame."""
    out = []
    for tw in sorted(set(det.tower_id.tolist())):
        idx = np.nonzero(det.tower_id == tw)[0]
        out.append(Detector(f"{det.name}.t{tw}", np.ascontiguousarray(det.xyz_mm[idx]),
                            np.ascontiguousarray(det.floor_id[idx]), np.ascontiguousarray(det.tower_id[idx])))
    return out


def split_stream(stream: Stream, det: Detector) -> list[Stream]:
    """An array's stream cut into per-tower streams (the PMT numbering of
    split_towers); a tower's PMTs must be contiguous in the array."""
    out = []
    for tw in sorted(set(det.tower_id.tolist())):
        idx = np.nonzero(det.tower_id == tw)[0]
        p0, p1 = int(idx[0]), int(idx[-1]) + 1
        if p1 - p0 != len(idx):
            raise ValueError("a tower's PMTs are not contiguous")
        a, b = int(stream.pmt_off[p0]), int(stream.pmt_off[p1])
        hits = stream.hits[a:b].copy()
        hits["pmt"] -= p0
        out.append(Stream(hits, (stream.pmt_off[p0:p1 + 1] - stream.pmt_off[p0]).astype(np.uint64)))
    return out


def stream_from_rows(rows, n_pmt: int) -> Stream:
    """(t, pmt, charge) rows in any order as a stream grouped by PMT, time
    order within a PMT (equal times keep their row order)."""
    hits = np.zeros(len(rows), HIT_DTYPE)
    for i, (t, p, q) in enumerate(rows):
        hits[i] = (t, p, q, 0)
    order = np.lexsort((np.arange(len(hits)), hits["t"], hits["pmt"]))
    hits = hits[order]
    off = np.zeros(n_pmt + 1, np.uint64)
    np.cumsum(np.bincount(hits["pmt"], minlength=n_pmt), out=off[1:])
    return Stream(hits, off)


# --------------------------------------------------------------- workloads

@dataclass
class Submission:
    """One slice as a producer hands it over: owned range [t0, t0 + S) plus
    the halos it includes (hits in [t0 - lead, t0 + S + HALO_NS))."""
    det_index: int
    t0: int
    stream: Stream


@dataclass
class Workload:
    name: str
    detectors: list[Detector]
    submissions: list[Submission]
    # per detector: the full stream the oracle sees (the multiset H of a run)
    runs: list[Stream] = field(default_factory=list)
    # per detector: slice t0 values of that detector, in submission order
    run_slices: list[list[int]] = field(default_factory=list)

    @property
    def n_hits(self) -> int:
        return sum(s.stream.n_hits for s in self.submissions)

    def owned_hits(self) -> int:
        n = 0
        for s in self.submissions:
            t = s.stream.hits["t"]
            n += int(np.count_nonzero((t >= s.t0) & (t < s.t0 + SLICE_NS)))
        return n


def _contiguous(det, det_index, n_slices, rate_hz, seed, stream, n_muons=0, n_bursts=0,
                slice_ns=SLICE_NS, t_origin=T_ORIGIN_NS, threads=None):
    """A run of n_slices contiguous slices; each submission carries both halos."""
    t_lo = t_origin - HALO_NS
    t_hi = t_origin + n_slices * slice_ns + HALO_NS
    full = gen_stream(det, t_lo, t_hi, rate_hz, n_muons=n_muons, n_bursts=n_bursts, seed=seed,
                      stream=stream, threads=threads)
    subs = []
    t0s = []
    for k in range(n_slices):
        t0 = t_origin + k * slice_ns
        subs.append(Submission(det_index, t0, cut(full, t0 - HALO_NS, t0 + slice_ns + HALO_NS)))
        t0s.append(t0)
    return full, subs, t0s


def cfg_nemo(seed: int = 0, threads=None) -> Workload:
    """NEMO Phase II tower, one 200 ms slice, 50 kHz background, 50 muons."""
    det = nemo_tower()
    full, subs, t0s = _contiguous(det, 0, 1, 50e3, seed, stream=1, n_muons=50, threads=threads)
    return Workload("nemo32_1slice", [det], subs, [full], [t0s])


def cfg_km3(seed: int = 0, threads=None) -> Workload:
    """KM3Net-It tower, 5 contiguous 200 ms slices, 55 kHz, 200 muons, one
    10 ms burst at 500 kHz on 3 PMTs per slice."""
    det = km3_tower()
    full, subs, t0s = _contiguous(det, 0, 5, 55e3, seed, stream=2, n_muons=200, n_bursts=5, threads=threads)
    return Workload("km3it84_5slices", [det], subs, [full], [t0s])


def cfg_batched(seed: int = 0, n_slices: int = 64, threads=None) -> Workload:
    """n independent slices (no halo) of 32- or 84-PMT towers, one rate per
    slice drawn from U[50, 500] kHz and applied to all its PMTs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dets = [nemo_tower(), km3_tower()]
    subs, runs, run_slices = [], [], []
    kinds = rng.integers(0, 2, n_slices)
    rates = rng.uniform(50e3, 500e3, n_slices)
    for k in range(n_slices):
        d = int(kinds[k])
        t0 = T_ORIGIN_NS + k * SLICE_NS
        st = gen_stream(dets[d], t0, t0 + SLICE_NS, float(rates[k]), seed=seed, stream=1000 + k,
                        threads=threads)
        subs.append(Submission(d, t0, st))
    return Workload(f"batched{n_slices}", dets, subs)


def cfg_scaled(seed: int = 0, threads=None) -> Workload:
    """32 towers of 84 PMTs (2688) on a 90 m grid, 55 kHz, one slice + halos, 1000 muons."""
    det = tower_array()
    full, subs, t0s = _contiguous(det, 0, 1, 55e3, seed, stream=4, n_muons=1000, threads=threads)
    return Workload("array2688_1slice", [det], subs, [full], [t0s])


def cfg_towers8(seed: int = 0, n_slices: int = 1, threads=None) -> Workload:
    """The eight KM3Net-It towers of the paper's proposed DAQ (84 PMTs each,
    4 x 2 on a 90 m grid) as eight detectors: contiguous 200 ms slices with
    halos at 55 kHz, 1000 muons per slice crossing the array.  Submission
    k * 8 + b is tower b's slice k; runs[b] is tower b's whole stream."""
    arr = tower_array(nx=4, ny=2)
    towers = split_towers(arr)
    full, subs, t0s = _contiguous(arr, 0, n_slices, 55e3, seed, stream=6, n_muons=1000 * n_slices,
                                  threads=threads)
    out = []
    for s in subs:
        for b, st in enumerate(split_stream(s.stream, arr)):
            out.append(Submission(b, s.t0, st))
    return Workload(f"towers8_{n_slices}slice", towers, out, split_stream(full, arr), [list(t0s) for _ in towers])


def cfg_serving_pool(seed: int = 0, slices_per_det: int = 20, threads=None,
                     dets: list[tuple[str, float]] | None = None) -> Workload:
    """Pre-generated slice pools of 4 detectors (32 @ 50 kHz, 84 @ 55 kHz,
    84 @ 55 kHz, 2688 @ 55 kHz); a replay rebases their timestamps."""
    spec = dets or [("nemo", 50e3), ("km3", 55e3), ("km3", 55e3), ("array", 55e3)]
    makers = {"nemo": nemo_tower, "km3": km3_tower, "array": tower_array}
    detectors, subs, runs, run_slices = [], [], [], []
    for i, (kind, rate) in enumerate(spec):
        det = makers[kind]()
        detectors.append(det)
        full, s, t0s = _contiguous(det, i, slices_per_det, rate, seed, stream=5000 + i,
                                   n_muons=10 * slices_per_det, threads=threads)
        subs += s
        runs.append(full)
        run_slices.append(t0s)
    return Workload("serving_pool", detectors, subs, runs, run_slices)


CONFIGS = {
    "nemo": cfg_nemo,
    "km3": cfg_km3,
    "batched": cfg_batched,
    "scaled": cfg_scaled,
    "towers8": cfg_towers8,
    "serving": cfg_serving_pool,
}

DEFAULT_PARAMS = dict(q_seed_adc=300, floor_tau_ns=20, tol_ns=20, n_num=6900, n_den=1499,
                      corr_window_ns=3000, threshold=4, win_half_ns=3000, slice_ns=SLICE_NS,
                      l0_hits=0, l0_window_ns=1000, l0_distinct_pmts=0,
                      seed_rule=0, sc_window_ns=20, fc_window_ns=100, afc_window_ns=250, sc_dist_mm=1000,
                      count_distinct_pmts=0)
