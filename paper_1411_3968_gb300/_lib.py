"""ctypes binding of libtrig.so (include/trig.h).  Argument marshalling only:
every step of the trigger runs in the library's CUDA kernels.  There is no
CPU fallback; loading fails loudly if the library is missing."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrig.so")

TRIG_OK = 0
TRIG_EINVAL = -1
TRIG_ENOMEM = -2
TRIG_EAGAIN = -3
TRIG_ETIMEOUT = -4
TRIG_EDEVICE = -5
TRIG_ECAPACITY = -6

TRIG_FLAG_BAD_PMT = 0x01
TRIG_FLAG_UNSORTED = 0x02
TRIG_FLAG_OUT_OF_RANGE = 0x04
TRIG_FLAG_TILE_FULL = 0x08
TRIG_FLAG_TRIG_FULL = 0x10
TRIG_FLAG_WIN_FULL = 0x20
TRIG_FLAG_TIMEOUT = 0x40
TRIG_FLAG_EV_FULL = 0x80
TRIG_EV_HALO_MAX = 8192

TRIG_RUN_GRAPH = 0x1
TRIG_RUN_TIMED = 0x2

HIT_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("charge", "<u2"), ("reserved", "<u4")])
TRIGGER_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("charge", "<u2"), ("count", "<u4")])
WINDOW_DTYPE = np.dtype([("lo", "<i8"), ("hi", "<i8"), ("n_hits", "<u8"), ("n_triggers", "<u8")])
STATS_DTYPE = np.dtype([("status", "<i4"), ("flags", "<u4"), ("n_hits", "<u8"), ("n_seeds", "<u8"),
                        ("n_triggers", "<u8"), ("n_windows", "<u8"), ("n_events", "<u8")])

TRACE_DTYPE = np.dtype([("slice_id", "<u8"), ("batch", "<u8"), ("batch_slices", "<u4"), ("n_pmt", "<u4"),
                        ("n_hits", "<u8"), ("status", "<i4"), ("continuation", "<u4"), ("t_submit_ns", "<i8"),
                        ("t_queued_ns", "<i8"), ("t_launch_ns", "<i8"), ("t_stats_ns", "<i8"), ("t_done_ns", "<i8"),
                        ("device_ms", "<f4"), ("copy_wait_us", "<u4")])

ASEED_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("tower", "<u2"), ("n_towers", "<u4")])
ASTATS_DTYPE = np.dtype([("n_tower_triggers", "<u8"), ("n_selected", "<u8"), ("n_windows", "<u8"),
                         ("n_hits", "<u8"), ("flags", "<u4"), ("status", "<i4")])
TRIG_AFLAG_SEED_FULL = 0x01
TRIG_AFLAG_WIN_FULL = 0x02
TRIG_AFLAG_HIT_FULL = 0x04
TRIG_AFLAG_TOWER_INCOMPLETE = 0x08

# symbols declared in include/trig.h and include/trig_array.h
EXPORTS = [
    "trig_create", "trig_destroy", "trig_detector_dtmax", "trig_detector_halo_ns", "trig_submit_slice",
    "trig_poll", "trig_result_free", "trig_engine_set_mode", "trig_engine_stats", "trig_last_error",
    "trig_batch_scratch_bytes", "trig_batch_run", "trig_slice_rows", "trig_set_tile_config",
    "trig_get_tile_config", "trig_kernel_launch_count", "trig_kernel_times", "trig_batch_run_noalloc",
    "trig_autotune", "trig_detector_tile_config", "trig_batch_events_scratch_bytes", "trig_batch_run_events",
    "trig_set_events", "trig_host_alloc", "trig_host_free", "trig_array_create", "trig_array_destroy", "trig_array_scratch_bytes", "trig_array_select",
    "trig_engine_hold", "trig_engine_set_staging_limit", "trig_engine_fail_result_allocs", "trig_set_device_wait",
    "trig_engine_trace", "trig_engine_trace_read",
]

NOALLOC_SCRATCH_BYTES = 64 << 20
NOALLOC_MAX_SLICES = 16


class TrigError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"trig error {code}: {msg}")
        self.code = code


class trig_geometry(ctypes.Structure):
    _fields_ = [("n_pmt", ctypes.c_uint32), ("xyz_mm", ctypes.c_void_p), ("floor_id", ctypes.c_void_p),
                ("tower_id", ctypes.c_void_p)]


class trig_params(ctypes.Structure):
    _fields_ = [("q_seed_adc", ctypes.c_uint32), ("floor_tau_ns", ctypes.c_uint32), ("tol_ns", ctypes.c_uint32),
                ("n_num", ctypes.c_uint32), ("n_den", ctypes.c_uint32), ("corr_window_ns", ctypes.c_uint32),
                ("threshold", ctypes.c_uint32), ("win_half_ns", ctypes.c_uint32), ("slice_ns", ctypes.c_int64),
                ("l0_hits", ctypes.c_uint32), ("l0_window_ns", ctypes.c_uint32), ("l0_distinct_pmts", ctypes.c_uint32),
                ("seed_rule", ctypes.c_uint32), ("sc_window_ns", ctypes.c_uint32),
                ("fc_window_ns", ctypes.c_uint32), ("afc_window_ns", ctypes.c_uint32),
                ("sc_dist_mm", ctypes.c_uint32), ("count_distinct_pmts", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class trig_result(ctypes.Structure):
    _fields_ = [("slice_id", ctypes.c_uint64), ("t0_ns", ctypes.c_int64), ("status", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("n_hits", ctypes.c_uint64), ("n_seeds", ctypes.c_uint64),
                ("n_triggers", ctypes.c_uint64), ("n_windows", ctypes.c_uint64), ("triggers", ctypes.c_void_p),
                ("windows", ctypes.c_void_p), ("latency_ns", ctypes.c_int64), ("events", ctypes.c_void_p),
                ("n_events", ctypes.c_uint64)]


class trig_slice_events(ctypes.Structure):
    _fields_ = [("events", ctypes.c_void_p), ("ev_cap", ctypes.c_uint64)]


class trig_tune_result(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_uint32), ("warps", ctypes.c_uint32), ("fill_pct", ctypes.c_uint32),
                ("n_tried", ctypes.c_uint32), ("ms", ctypes.c_double)]


class trig_slice_dev(ctypes.Structure):
    _fields_ = [("det", ctypes.c_void_p), ("hits", ctypes.c_void_p), ("pmt_off", ctypes.c_void_p),
                ("n_hits", ctypes.c_uint64), ("t0_ns", ctypes.c_int64), ("triggers", ctypes.c_void_p),
                ("trig_cap", ctypes.c_uint64), ("windows", ctypes.c_void_p), ("win_cap", ctypes.c_uint64),
                ("stats", ctypes.c_void_p)]


class trig_array_params(ctypes.Structure):
    _fields_ = [("min_towers", ctypes.c_uint32), ("corr_window_ns", ctypes.c_uint32),
                ("win_half_ns", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class trig_array_out(ctypes.Structure):
    _fields_ = [("seeds", ctypes.c_void_p), ("seed_cap", ctypes.c_uint64), ("windows", ctypes.c_void_p),
                ("win_cap", ctypes.c_uint64), ("frag_off", ctypes.c_void_p), ("hits", ctypes.c_void_p),
                ("hit_cap", ctypes.c_uint64), ("stats", ctypes.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load libtrig.so (built by __graft_entry__.build() or build.build());
    the environment variable TRIG_LIB names another build of it (a checked
    or instrumented one)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or os.environ.get("TRIG_LIB") or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libtrig.so not built at {p}; run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    c = ctypes
    sig = {
        "trig_create": (c.c_int, [c.POINTER(trig_geometry), c.POINTER(trig_params), c.POINTER(c.c_void_p)]),
        "trig_destroy": (c.c_int, [c.c_void_p]),
        "trig_detector_dtmax": (c.c_int, [c.c_void_p, c.c_void_p]),
        "trig_detector_halo_ns": (c.c_int64, [c.c_void_p]),
        "trig_submit_slice": (c.c_int, [c.c_void_p, c.c_int64, c.c_void_p, c.c_void_p, c.c_int,
                                        c.POINTER(c.c_uint64)]),
        "trig_poll": (c.c_int, [c.c_void_p, c.c_int, c.POINTER(c.POINTER(trig_result))]),
        "trig_result_free": (None, [c.POINTER(trig_result)]),
        "trig_engine_set_mode": (c.c_int, [c.c_int]),
        "trig_engine_stats": (c.c_int, [c.POINTER(c.c_uint64), c.POINTER(c.c_uint64)]),
        "trig_engine_hold": (c.c_int, [c.c_int]),
        "trig_engine_set_staging_limit": (c.c_int, [c.c_uint64]),
        "trig_engine_fail_result_allocs": (c.c_int, [c.c_uint32]),
        "trig_set_device_wait": (c.c_int, [c.c_uint64, c.c_int]),
        "trig_engine_trace": (c.c_int, [c.c_uint32]),
        "trig_engine_trace_read": (c.c_int, [c.c_void_p, c.c_uint32, c.POINTER(c.c_uint32)]),
        "trig_last_error": (c.c_char_p, []),
        "trig_batch_scratch_bytes": (c.c_size_t, [c.POINTER(trig_slice_dev), c.c_uint32]),
        "trig_batch_run": (c.c_int, [c.POINTER(trig_slice_dev), c.c_uint32, c.c_void_p, c.c_size_t, c.c_void_p,
                                     c.c_uint32]),
        "trig_slice_rows": (c.c_int, [c.POINTER(trig_slice_dev), c.c_void_p, c.c_void_p, c.POINTER(c.c_uint64),
                                      c.c_void_p, c.c_size_t, c.c_void_p]),
        "trig_set_tile_config": (c.c_int, [c.c_uint32, c.c_uint32, c.c_uint32]),
        "trig_get_tile_config": (c.c_int, [c.POINTER(c.c_uint32), c.POINTER(c.c_uint32), c.POINTER(c.c_uint32)]),
        "trig_autotune": (c.c_int, [c.c_void_p, c.POINTER(trig_slice_dev), c.c_uint32, c.c_void_p,
                                    c.POINTER(trig_tune_result)]),
        "trig_detector_tile_config": (c.c_int, [c.c_void_p, c.POINTER(c.c_uint32), c.POINTER(c.c_uint32),
                                                c.POINTER(c.c_uint32)]),
        "trig_kernel_launch_count": (c.c_uint64, []),
        "trig_batch_run_noalloc": (c.c_int, [c.POINTER(trig_slice_dev), c.c_uint32, c.c_void_p]),
        "trig_kernel_times": (c.c_int, [c.POINTER(c.c_double), c.POINTER(c.c_char_p), c.c_uint32,
                                        c.POINTER(c.c_uint32)]),
        "trig_batch_events_scratch_bytes": (c.c_size_t, [c.POINTER(trig_slice_dev), c.POINTER(trig_slice_events),
                                                         c.c_uint32]),
        "trig_batch_run_events": (c.c_int, [c.POINTER(trig_slice_dev), c.POINTER(trig_slice_events), c.c_uint32,
                                            c.c_void_p, c.c_size_t, c.c_void_p, c.c_uint32]),
        "trig_set_events": (c.c_int, [c.c_void_p, c.c_int]),
        "trig_host_alloc": (c.c_int, [c.c_size_t, c.POINTER(c.c_void_p)]),
        "trig_host_free": (c.c_int, [c.c_void_p]),
        "trig_array_create": (c.c_int, [c.POINTER(c.c_void_p), c.c_uint32, c.POINTER(trig_array_params),
                                        c.POINTER(c.c_void_p)]),
        "trig_array_destroy": (c.c_int, [c.c_void_p]),
        "trig_array_scratch_bytes": (c.c_size_t, [c.c_void_p, c.POINTER(trig_slice_dev), c.POINTER(trig_array_out)]),
        "trig_array_select": (c.c_int, [c.c_void_p, c.POINTER(trig_slice_dev), c.POINTER(trig_array_out), c.c_void_p,
                                        c.c_size_t, c.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != TRIG_OK:
        raise TrigError(rc, load().trig_last_error().decode())
    return rc


def trig_last_error() -> str:
    return load().trig_last_error().decode()


# ------------------------------------------------------------------ detectors

class Detector:
    """Owns a trig_detector handle."""

    def __init__(self, xyz_mm, floor_id, params: dict, tower_id=None):
        lib = load()
        self.xyz = np.ascontiguousarray(xyz_mm, np.int32).reshape(-1, 3)
        self.floor_id = np.ascontiguousarray(floor_id, np.uint32)
        self.tower_id = None if tower_id is None else np.ascontiguousarray(tower_id, np.uint32)
        self.n_pmt = self.xyz.shape[0]
        self.params = dict(params)
        g = trig_geometry(self.n_pmt, self.xyz.ctypes.data, self.floor_id.ctypes.data,
                          None if self.tower_id is None else self.tower_id.ctypes.data)
        p = trig_params(*(int(params.get(f, 0)) for f, _ in trig_params._fields_))
        h = ctypes.c_void_p()
        _check(lib.trig_create(ctypes.byref(g), ctypes.byref(p), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            load().trig_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def halo_ns(self) -> int:
        return int(load().trig_detector_halo_ns(self.handle))

    def dtmax(self) -> np.ndarray:
        out = np.empty((self.n_pmt, self.n_pmt), np.int32)
        _check(load().trig_detector_dtmax(self.handle, out.ctypes.data))
        return out


def trig_create(xyz_mm, floor_id, params, tower_id=None) -> Detector:
    return Detector(xyz_mm, floor_id, params, tower_id)


def trig_destroy(det: Detector) -> None:
    det.close()


# --------------------------------------------------------------------- engine

def trig_submit_slice(det: Detector, t0: int, hits: np.ndarray, pmt_off: np.ndarray, is_continuation: int = 0) -> int:
    h = np.ascontiguousarray(hits, HIT_DTYPE)
    o = np.ascontiguousarray(pmt_off, np.uint64)
    sid = ctypes.c_uint64()
    rc = load().trig_submit_slice(det.handle, int(t0), h.ctypes.data if len(h) else None, o.ctypes.data,
                                  int(is_continuation), ctypes.byref(sid))
    _check(rc)
    return int(sid.value)


class _Owner:
    """Frees a trig_result when the last array viewing it is gone."""

    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        try:
            load().trig_result_free(self.ptr)
        except Exception:
            pass


class _View:
    """Numpy view of library memory (read-only unless stated) that keeps its
    owner alive."""

    def __init__(self, owner, addr, n, dtype, readonly=True):
        self.owner = owner
        self.__array_interface__ = {"shape": (n,), "typestr": dtype.str, "descr": dtype.descr,
                                    "data": (addr, readonly), "version": 3}


def _view(owner, ptr, n, dtype):
    n = int(n)
    if n == 0 or not ptr:
        return np.empty(0, dtype)
    return np.asarray(_View(owner, ptr, n, dtype)).view(dtype)


class Result:
    """One slice's result.  Its arrays are read-only views of the library's
    result memory (no copy), released once the Result and every array taken
    from it are gone."""

    def __init__(self, ptr):
        r = ptr.contents
        owner = _Owner(ptr)
        self.slice_id = int(r.slice_id)
        self.t0 = int(r.t0_ns)
        self.status = int(r.status)
        self.flags = int(r.flags)
        self.n_hits = int(r.n_hits)
        self.n_seeds = int(r.n_seeds)
        self.latency_ns = int(r.latency_ns)
        self.triggers = _view(owner, r.triggers, r.n_triggers, TRIGGER_DTYPE)
        self.windows = _view(owner, r.windows, r.n_windows, WINDOW_DTYPE)
        self.n_events = int(r.n_events)
        self.events = _view(owner, r.events, r.n_events if r.events else 0, HIT_DTYPE)
        self._owner = owner


def _copy(ptr, n, dtype):
    n = int(n)
    if n == 0 or not ptr:
        return np.empty(0, dtype)
    buf = (ctypes.c_char * (n * dtype.itemsize)).from_address(ptr)
    return np.frombuffer(buf, dtype).copy()


def trig_poll(det: Detector, timeout_ms: int = -1) -> Result | None:
    lib = load()
    out = ctypes.POINTER(trig_result)()
    rc = lib.trig_poll(det.handle, int(timeout_ms), ctypes.byref(out))
    if rc == TRIG_EAGAIN:
        return None
    _check(rc)
    return Result(out)


class _HostBlock:
    """Page-locked host memory from trig_host_alloc, freed with the last
    array viewing it."""

    def __init__(self, nbytes: int):
        p = ctypes.c_void_p()
        _check(load().trig_host_alloc(int(nbytes), ctypes.byref(p)))
        self.ptr = p.value

    def __del__(self):
        try:
            if self.ptr:
                load().trig_host_free(ctypes.c_void_p(self.ptr))
                self.ptr = None
        except Exception:
            pass


def pinned_copy(a: np.ndarray) -> np.ndarray:
    """A copy of `a` in page-locked host memory (trig_host_alloc): slices
    submitted from it reach the device by DMA."""
    a = np.ascontiguousarray(a)
    if a.nbytes == 0:
        return a.copy()
    blk = _HostBlock(a.nbytes)
    out = np.asarray(_View(blk, blk.ptr, a.nbytes, np.dtype(np.uint8), readonly=False)).view(a.dtype).reshape(a.shape)
    np.copyto(out, a)
    return out


def trig_set_events(det: "Detector", on: bool = True) -> None:
    """Engine results of det's later submissions carry the event payload."""
    _check(load().trig_set_events(det.handle, 1 if on else 0))


def trig_engine_set_mode(mode: int) -> None:
    _check(load().trig_engine_set_mode(int(mode)))


def trig_engine_stats() -> tuple[int, int]:
    b, s = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().trig_engine_stats(ctypes.byref(b), ctypes.byref(s)))
    return int(b.value), int(s.value)


def trig_engine_hold(on: bool) -> None:
    """Admit no new engine batch while on (submissions still queue)."""
    _check(load().trig_engine_hold(1 if on else 0))


def trig_engine_set_staging_limit(nbytes: int) -> None:
    """Device staging memory the engine's submissions may hold (0: no limit)."""
    _check(load().trig_engine_set_staging_limit(int(nbytes)))


def trig_engine_fail_result_allocs(n: int) -> None:
    """Failure injection: the next n result-memory requests fail (TRIG_ENOMEM results)."""
    _check(load().trig_engine_fail_result_allocs(int(n)))


def trig_engine_trace(capacity: int) -> None:
    """Start recording per-slice engine records (0 stops)."""
    _check(load().trig_engine_trace(int(capacity)))


def trig_engine_trace_read(max_records: int = 1 << 20) -> np.ndarray:
    """The recorded slices so far (TRACE_DTYPE), oldest first; they are
    removed from the engine's record."""
    out = np.zeros(int(max_records), TRACE_DTYPE)
    n = ctypes.c_uint32()
    _check(load().trig_engine_trace_read(out.ctypes.data, len(out), ctypes.byref(n)))
    return out[: n.value].copy()


def trig_set_device_wait(limit_ns: int = 0, stall: bool = False) -> None:
    """Limit of the tile pass's device waits (0: the default second); stall
    is the test control that stages nothing, so the waits run out."""
    _check(load().trig_set_device_wait(int(limit_ns), 1 if stall else 0))


def trig_set_tile_config(cap: int, warps: int, fill_pct: int) -> None:
    _check(load().trig_set_tile_config(int(cap), int(warps), int(fill_pct)))


def trig_get_tile_config() -> tuple[int, int, int]:
    c, w, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().trig_get_tile_config(ctypes.byref(c), ctypes.byref(w), ctypes.byref(f)))
    return int(c.value), int(w.value), int(f.value)


def trig_autotune(det: "Detector", slices, stream_ptr: int = 0) -> dict:
    """Tune det's launch shape on device-resident slices of det."""
    arr = _array(slices)
    r = trig_tune_result()
    _check(load().trig_autotune(det.handle, arr, len(slices), stream_ptr or None, ctypes.byref(r)))
    return {"cap": r.cap, "warps": r.warps, "fill_pct": r.fill_pct, "n_tried": r.n_tried, "ms": r.ms}


def trig_detector_tile_config(det: "Detector") -> dict:
    c, w, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    t = load().trig_detector_tile_config(det.handle, ctypes.byref(c), ctypes.byref(w), ctypes.byref(f))
    if t < 0:
        _check(t)
    return {"cap": int(c.value), "warps": int(w.value), "fill_pct": int(f.value), "tuned": bool(t)}


def trig_kernel_launch_count() -> int:
    return int(load().trig_kernel_launch_count())


def trig_kernel_times() -> tuple[dict, int]:
    """Average ms per pipeline kernel over the TIMED runs since the last call."""
    ms = (ctypes.c_double * 16)()
    names = (ctypes.c_char_p * 16)()
    nr = ctypes.c_uint32()
    k = load().trig_kernel_times(ms, names, 16, ctypes.byref(nr))
    if k < 0:
        _check(k)
    return {names[i].decode(): float(ms[i]) for i in range(k)}, int(nr.value)


# ------------------------------------------------------------- device batches

def slice_dev(det: Detector, hits_ptr: int, pmt_off_ptr: int, n_hits: int, t0: int, trig_ptr: int, trig_cap: int,
              win_ptr: int, win_cap: int, stats_ptr: int) -> trig_slice_dev:
    return trig_slice_dev(det.handle.value, hits_ptr, pmt_off_ptr, n_hits, t0, trig_ptr, trig_cap, win_ptr, win_cap,
                          stats_ptr)


def _array(slices):
    arr = (trig_slice_dev * len(slices))(*slices)
    return arr


def trig_batch_scratch_bytes(slices) -> int:
    arr = _array(slices)
    n = load().trig_batch_scratch_bytes(arr, len(slices))
    if n == 0:
        raise TrigError(TRIG_EINVAL, trig_last_error())
    return int(n)


def trig_batch_run(slices, scratch_ptr: int, scratch_bytes: int, stream_ptr: int = 0, flags: int = 0) -> None:
    arr = _array(slices)
    _check(load().trig_batch_run(arr, len(slices), scratch_ptr, scratch_bytes, stream_ptr or None, flags))


def _events_array(events):
    return (trig_slice_events * len(events))(*events)


def trig_batch_events_scratch_bytes(slices, events) -> int:
    n = load().trig_batch_events_scratch_bytes(_array(slices), _events_array(events), len(slices))
    if n == 0:
        raise TrigError(TRIG_EINVAL, trig_last_error())
    return int(n)


def trig_batch_run_events(slices, events, scratch_ptr: int, scratch_bytes: int, stream_ptr: int = 0,
                          flags: int = 0) -> None:
    _check(load().trig_batch_run_events(_array(slices), _events_array(events), len(slices), scratch_ptr,
                                        scratch_bytes, stream_ptr or None, flags))


def trig_batch_run_noalloc(slices, stream_ptr: int) -> None:
    """trig_batch_run on the library's static scratch (no allocation), on a
    stream the caller created (the legacy default stream is refused)."""
    arr = _array(slices)
    _check(load().trig_batch_run_noalloc(arr, len(slices), stream_ptr or None))


def trig_slice_rows(s: trig_slice_dev, merged_ptr: int, seedcnt_ptr: int, scratch_ptr: int, scratch_bytes: int,
                    stream_ptr: int = 0) -> int:
    n = ctypes.c_uint64()
    _check(load().trig_slice_rows(ctypes.byref(s), merged_ptr, seedcnt_ptr, ctypes.byref(n), scratch_ptr,
                                  scratch_bytes, stream_ptr or None))
    return int(n.value)


def win_cap_for(params: dict) -> int:
    """A window capacity that can never overflow for one slice."""
    h = int(params["win_half_ns"])
    return (int(params["slice_ns"]) + 2 * h) // (2 * h + 2) + 2


# ------------------------------------------------------- multi-tower selection

class Array:
    """Towers grouped for the cross-tower selection (trig_array_create)."""

    def __init__(self, towers: list, min_towers: int = 2, corr_window_ns: int = 3000, win_half_ns: int = 3000):
        self.towers = list(towers)
        self.params = dict(min_towers=min_towers, corr_window_ns=corr_window_ns, win_half_ns=win_half_ns)
        arr = (ctypes.c_void_p * len(self.towers))(*[t.handle.value for t in self.towers])
        p = trig_array_params(int(min_towers), int(corr_window_ns), int(win_half_ns), 0)
        h = ctypes.c_void_p()
        _check(load().trig_array_create(arr, len(self.towers), ctypes.byref(p), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle and self.handle.value:
            load().trig_array_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trig_array_scratch_bytes(array: Array, slices, out: trig_array_out) -> int:
    n = load().trig_array_scratch_bytes(array.handle, _array(slices), ctypes.byref(out))
    if n == 0:
        raise TrigError(TRIG_EINVAL, trig_last_error())
    return int(n)


def trig_array_select(array: Array, slices, out: trig_array_out, scratch_ptr: int, scratch_bytes: int,
                      stream_ptr: int = 0) -> None:
    _check(load().trig_array_select(array.handle, _array(slices), ctypes.byref(out), scratch_ptr, scratch_bytes,
                                    stream_ptr or None))
