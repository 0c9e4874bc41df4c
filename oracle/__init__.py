"""CPU oracle of the online muon trigger -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (``paper_1411_3968_gb300``) never does, and shares no code with it.

Python face of ``oracle.c`` (plain C, compiled with gcc on first use):

* ``dtmax(det, params)``   exact-integer causality table dt_max[i][j]
  (unclamped), following the "Muon trigger strategy" section's time-space
  correlation with the constants given as parameters.
* ``merge(hits)``          hits ordered by (t, pmt, charge) -- the Hit
  Manager's time-ordered merge ("DAQ system of NEMO Phase II").
* ``run(det, params, hits, slice_t0s)``  seeds with counts, triggers and
  merged windows per slice ("Sorting and triggering in GPU").
* ``events(hits, windows)``  the event payload: the hits inside a slice's
  merged windows, in (t, pmt, charge) order.
* ``oracle.array.select(...)``  the multi-tower selection and window
  readback ("Results and perspectives"), numpy over the towers' triggers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HIT_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("charge", "<u2"), ("reserved", "<u4")])
SEED_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("charge", "<u2"), ("count", "<u4")])
WINDOW_DTYPE = np.dtype([("lo", "<i8"), ("hi", "<i8"), ("n_hits", "<u8"), ("n_triggers", "<u8")])

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with plain gcc -O2."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, src, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("q_seed_adc", ctypes.c_uint32),
        ("floor_tau_ns", ctypes.c_uint32),
        ("tol_ns", ctypes.c_uint32),
        ("n_num", ctypes.c_uint32),
        ("n_den", ctypes.c_uint32),
        ("corr_window_ns", ctypes.c_uint32),
        ("threshold", ctypes.c_uint32),
        ("win_half_ns", ctypes.c_uint32),
        ("slice_ns", ctypes.c_int64),
        ("l0_hits", ctypes.c_uint32),
        ("l0_window_ns", ctypes.c_uint32),
        ("l0_distinct_pmts", ctypes.c_uint32),
        ("seed_rule", ctypes.c_uint32),
        ("sc_window_ns", ctypes.c_uint32),
        ("fc_window_ns", ctypes.c_uint32),
        ("afc_window_ns", ctypes.c_uint32),
        ("sc_dist_mm", ctypes.c_uint32),
        ("count_distinct_pmts", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class _SliceResult(ctypes.Structure):
    _fields_ = [
        ("n_seeds", ctypes.c_uint64),
        ("n_triggers", ctypes.c_uint64),
        ("n_windows", ctypes.c_uint64),
        ("seeds", ctypes.c_void_p),
        ("triggers", ctypes.c_void_p),
        ("windows", ctypes.c_void_p),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_dtmax_pair.restype = ctypes.c_int64
        lib.oracle_dtmax_pair.argtypes = [ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.oracle_dtmax.restype = ctypes.c_int
        lib.oracle_dtmax.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_void_p]
        lib.oracle_merge.restype = ctypes.c_int
        lib.oracle_merge.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(_Params),
                                   ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint32,
                                   ctypes.c_int, ctypes.POINTER(_SliceResult)]
        lib.oracle_free.restype = None
        lib.oracle_free.argtypes = [ctypes.POINTER(_SliceResult), ctypes.c_uint32]
        lib.oracle_threads_used.restype = ctypes.c_int
        lib.oracle_threads_used.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _params(p: dict) -> _Params:
    s = _Params()
    for name, _ in _Params._fields_:
        setattr(s, name, int(p.get(name, 0)))
    return s


def dtmax_pair(d2_mm2: int, tol_ns=20, n_num=6900, n_den=1499) -> int:
    return int(_load().oracle_dtmax_pair(int(d2_mm2), tol_ns, n_num, n_den))


def dtmax(xyz_mm: np.ndarray, params: dict) -> np.ndarray:
    """Exact (unclamped) dt_max table, int32 [P, P]."""
    xyz = np.ascontiguousarray(xyz_mm, np.int32)
    P = xyz.shape[0]
    out = np.empty((P, P), np.int32)
    rc = _load().oracle_dtmax(P, xyz.ctypes.data, params["tol_ns"], params["n_num"], params["n_den"],
                              out.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_dtmax failed ({rc})")
    return out


def merge(hits: np.ndarray) -> np.ndarray:
    """Hits ordered by (t, pmt, charge); equal keys keep input order."""
    h = np.ascontiguousarray(hits, HIT_DTYPE)
    out = np.empty_like(h)
    rc = _load().oracle_merge(h.ctypes.data, len(h), out.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_merge failed ({rc})")
    return out


@dataclass
class SliceResult:
    t0: int
    seeds: np.ndarray       # SEED_DTYPE, every seed with its causal count
    triggers: np.ndarray    # SEED_DTYPE, seeds with count >= threshold
    windows: np.ndarray     # WINDOW_DTYPE


def run(xyz_mm, floor_id, params: dict, hits: np.ndarray, slice_t0s, threads: int = 0,
        tower_id=None) -> list[SliceResult]:
    """Trigger every slice [t0, t0 + slice_ns) against the whole hit set.
    tower_id (per PMT, optional) groups floors into towers for the
    consecutive-floor coincidence; None puts every floor in one tower."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz_mm, np.int32)
    fl = np.ascontiguousarray(floor_id, np.uint32)
    tw = None if tower_id is None else np.ascontiguousarray(tower_id, np.uint32)
    h = np.ascontiguousarray(hits, HIT_DTYPE)
    t0s = np.ascontiguousarray(np.asarray(slice_t0s, np.int64))
    n = len(t0s)
    res = (_SliceResult * max(n, 1))()
    par = _params(params)
    rc = lib.oracle_run(xyz.shape[0], xyz.ctypes.data, fl.ctypes.data, None if tw is None else tw.ctypes.data,
                        ctypes.byref(par), h.ctypes.data,
                        len(h), t0s.ctypes.data, n, int(threads), res)
    if rc:
        raise RuntimeError(f"oracle_run failed ({rc})")
    out = []
    try:
        for k in range(n):
            r = res[k]
            seeds = _copy(r.seeds, r.n_seeds, SEED_DTYPE)
            trig = _copy(r.triggers, r.n_triggers, SEED_DTYPE)
            win = _copy(r.windows, r.n_windows, WINDOW_DTYPE)
            out.append(SliceResult(int(t0s[k]), seeds, trig, win))
    finally:
        lib.oracle_free(res, n)
    return out


def events(hits: np.ndarray, windows: np.ndarray) -> np.ndarray:
    """The event payload of a slice ("DAQ system of NEMO Phase II": the
    window around each trigger seed is stored; "Sorting and triggering in
    GPU": all hits within +-3 us of a seed are tagged and sent back): every
    hit with lo <= t <= hi for one of the slice's merged windows, ordered by
    (t, pmt, charge).  The windows are disjoint and time-ordered, so a hit
    belongs to the last window whose lo is <= t, if t <= that window's hi."""
    h = merge(hits)
    if len(windows) == 0 or len(h) == 0:
        return h[:0]
    k = np.searchsorted(windows["lo"], h["t"], side="right") - 1
    inside = (k >= 0) & (h["t"] <= windows["hi"][np.maximum(k, 0)])
    return h[inside]


def threads_used(threads: int = 0) -> int:
    return int(_load().oracle_threads_used(int(threads)))


def _copy(ptr, n, dtype):
    n = int(n)
    if n == 0 or not ptr:
        return np.empty(0, dtype)
    buf = (ctypes.c_char * (n * dtype.itemsize)).from_address(ptr)
    return np.frombuffer(bytes(buf), dtype).copy()
