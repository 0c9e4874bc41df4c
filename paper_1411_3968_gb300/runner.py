"""Device-resident batches: PyTorch holds the device memory and the stream,
libtrig.so does all the work (trig_batch_run / trig_slice_rows)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import ASEED_DTYPE, ASTATS_DTYPE, HIT_DTYPE, STATS_DTYPE, TRIGGER_DTYPE, WINDOW_DTYPE


def _dev_bytes(nbytes: int, device) -> torch.Tensor:
    # 256-byte aligned allocation (the caching allocator aligns to >= 512 B)
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def _to_dev(a: np.ndarray, device) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1))
    out = _dev_bytes(t.numel(), device)
    if t.numel():
        out[: t.numel()].copy_(t)
    return out


@dataclass
class SliceIn:
    det: "_lib.Detector"
    t0: int
    hits: np.ndarray        # HIT_DTYPE, grouped by PMT
    pmt_off: np.ndarray     # uint64, n_pmt + 1


class DeviceBatch:
    """Inputs resident in HBM, outputs and scratch pre-allocated; run()
    enqueues the whole hot path for all slices on the current stream."""

    def __init__(self, slices: list[SliceIn], device="cuda", trig_cap: int | None = None, events: bool = False):
        self.slices = slices
        self.device = torch.device(device)
        self.hits = [_to_dev(s.hits, self.device) for s in slices]
        self.offs = [_to_dev(np.asarray(s.pmt_off, np.uint64), self.device) for s in slices]
        self.trig_cap = [max(1, len(s.hits) if trig_cap is None else trig_cap) for s in slices]
        self.win_cap = [_lib.win_cap_for(s.det.params) for s in slices]
        self.trig = [_dev_bytes(c * TRIGGER_DTYPE.itemsize, self.device) for c in self.trig_cap]
        self.win = [_dev_bytes(c * WINDOW_DTYPE.itemsize, self.device) for c in self.win_cap]
        self.stats = _dev_bytes(len(slices) * STATS_DTYPE.itemsize, self.device)
        self.descs = []
        for i, s in enumerate(slices):
            self.descs.append(_lib.slice_dev(s.det, self.hits[i].data_ptr(), self.offs[i].data_ptr(), len(s.hits),
                                             int(s.t0), self.trig[i].data_ptr(), self.trig_cap[i],
                                             self.win[i].data_ptr(), self.win_cap[i],
                                             self.stats.data_ptr() + i * STATS_DTYPE.itemsize))
        # optional event outputs (all hits inside the merged windows)
        self.events = None
        if events:
            self._alloc_events()
        self.scratch_bytes = self._scratch_need()
        self.scratch = _dev_bytes(self.scratch_bytes + 256, self.device)
        self.n_hits = sum(len(s.hits) for s in slices)
        self.input_bytes = sum(s.hits.nbytes + np.asarray(s.pmt_off).nbytes for s in slices)

    def _alloc_events(self) -> None:
        self.ev_cap = [max(1, len(s.hits)) for s in self.slices]
        self.ev = [_dev_bytes(c * HIT_DTYPE.itemsize, self.device) for c in self.ev_cap]
        self.events = [_lib.trig_slice_events(self.ev[i].data_ptr(), self.ev_cap[i]) for i in range(len(self.slices))]

    def set_events(self, on: bool) -> None:
        """Turns event extraction on (buffers of one entry per hit) or off
        for later runs of the same resident slices."""
        if on and self.events is None:
            self._alloc_events()
        elif not on:
            self.events = None
            self.ev = None

    def _scratch_need(self) -> int:
        if self.events is not None:
            return _lib.trig_batch_events_scratch_bytes(self.descs, self.events)
        return _lib.trig_batch_scratch_bytes(self.descs)

    def ensure_scratch(self) -> None:
        """Grows the scratch when the batch plan needs more, e.g. after the
        autotuner changed a detector's tile shape."""
        need = self._scratch_need()
        if need > self.scratch_bytes:
            self.scratch = _dev_bytes(need + 256, self.device)
            self.scratch_bytes = need

    def run(self, graph: bool = False, stream=None, timed: bool = False) -> None:
        self.ensure_scratch()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        flags = (_lib.TRIG_RUN_GRAPH if graph else 0) | (_lib.TRIG_RUN_TIMED if timed else 0)
        if self.events is not None:
            _lib.trig_batch_run_events(self.descs, self.events, self.scratch.data_ptr(), self.scratch_bytes,
                                       st.cuda_stream, flags)
        else:
            _lib.trig_batch_run(self.descs, self.scratch.data_ptr(), self.scratch_bytes, st.cuda_stream, flags)

    def run_each(self, stream=None) -> None:
        """Plain per-slice launches: one launch sequence per slice."""
        self.ensure_scratch()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        for d in self.descs:
            _lib.trig_batch_run([d], self.scratch.data_ptr(), self.scratch_bytes, st.cuda_stream, 0)

    def results(self):
        torch.cuda.synchronize(self.device)
        stats = np.frombuffer(self.stats.cpu().numpy().tobytes()[: len(self.slices) * STATS_DTYPE.itemsize],
                              STATS_DTYPE).copy()
        out = []
        for i in range(len(self.slices)):
            nt = min(int(stats[i]["n_triggers"]), self.trig_cap[i])
            nw = min(int(stats[i]["n_windows"]), self.win_cap[i])
            trig = np.frombuffer(self.trig[i][: nt * TRIGGER_DTYPE.itemsize].cpu().numpy().tobytes(), TRIGGER_DTYPE)
            win = np.frombuffer(self.win[i][: nw * WINDOW_DTYPE.itemsize].cpu().numpy().tobytes(), WINDOW_DTYPE)
            out.append((stats[i], trig.copy(), win.copy()))
        return out

    def event_hits(self):
        """Per slice: the event payload (hits inside the merged windows, in
        (t, pmt, charge) order) and n_events; run() must have been called."""
        torch.cuda.synchronize(self.device)
        stats = np.frombuffer(self.stats.cpu().numpy().tobytes()[: len(self.slices) * STATS_DTYPE.itemsize],
                              STATS_DTYPE).copy()
        out = []
        for i in range(len(self.slices)):
            ne = int(stats[i]["n_events"])
            full = bool(stats[i]["flags"] & _lib.TRIG_FLAG_EV_FULL)
            k = 0 if full else min(ne, self.ev_cap[i])
            ev = np.frombuffer(self.ev[i][: k * HIT_DTYPE.itemsize].cpu().numpy().tobytes(), HIT_DTYPE).copy()
            out.append((ev, ne, full))
        return out

    def rows(self, i: int):
        """Merged owned hits of slice i and their seed counts (0xFFFFFFFF: not a seed)."""
        s = self.slices[i]
        n = max(len(s.hits), 1)
        merged = _dev_bytes(n * HIT_DTYPE.itemsize, self.device)
        seedcnt = _dev_bytes(n * 4, self.device)
        self.ensure_scratch()
        st = torch.cuda.current_stream(self.device)
        n_owned = _lib.trig_slice_rows(self.descs[i], merged.data_ptr(), seedcnt.data_ptr(), self.scratch.data_ptr(),
                                       self.scratch_bytes, st.cuda_stream)
        m = np.frombuffer(merged[: n_owned * HIT_DTYPE.itemsize].cpu().numpy().tobytes(), HIT_DTYPE).copy()
        c = np.frombuffer(seedcnt[: n_owned * 4].cpu().numpy().tobytes(), np.uint32).copy()
        return m, c


class ArrayBatch:
    """The towers' slices of one period resident in HBM; run() enqueues each
    tower's trigger (one trig_batch_run over the towers) and then the
    cross-tower selection with the window readback (trig_array_select) on
    one stream.  slices[b] must be tower b of `array`."""

    def __init__(self, array: "_lib.Array", slices: list[SliceIn], device="cuda", seed_cap: int | None = None,
                 win_cap: int | None = None, hit_cap: int | None = None):
        self.array = array
        self.batch = DeviceBatch(slices, device=device)
        dev = self.batch.device
        nt = len(slices)
        n_trig = sum(self.batch.trig_cap)
        h = int(array.params["win_half_ns"])
        span = int(slices[0].det.params["slice_ns"]) + 2 * h
        self.seed_cap = max(1, n_trig if seed_cap is None else seed_cap)
        self.win_cap = max(1, min(n_trig, span // (2 * h + 2) + 1) if win_cap is None else win_cap)
        self.hit_cap = max(1, self.batch.n_hits if hit_cap is None else hit_cap)
        self.seeds = _dev_bytes(self.seed_cap * ASEED_DTYPE.itemsize, dev)
        self.windows = _dev_bytes(self.win_cap * WINDOW_DTYPE.itemsize, dev)
        self.frag_off = _dev_bytes((self.win_cap * nt + 1) * 8, dev)
        self.hits = _dev_bytes(self.hit_cap * HIT_DTYPE.itemsize, dev)
        self.stats = _dev_bytes(ASTATS_DTYPE.itemsize, dev)
        self.out = _lib.trig_array_out(self.seeds.data_ptr(), self.seed_cap, self.windows.data_ptr(), self.win_cap,
                                       self.frag_off.data_ptr(), self.hits.data_ptr(), self.hit_cap,
                                       self.stats.data_ptr())
        self.scratch_bytes = _lib.trig_array_scratch_bytes(array, self.batch.descs, self.out)
        self.scratch = _dev_bytes(self.scratch_bytes + 256, dev)
        self.n_towers = nt

    def run(self, graph: bool = False, stream=None) -> None:
        st = stream if stream is not None else torch.cuda.current_stream(self.batch.device)
        self.batch.run(graph=graph, stream=st)
        self.select(st)

    def select(self, stream=None) -> None:
        """The selection and readback alone, on the towers' last results."""
        st = stream if stream is not None else torch.cuda.current_stream(self.batch.device)
        _lib.trig_array_select(self.array, self.batch.descs, self.out, self.scratch.data_ptr(), self.scratch_bytes,
                               st.cuda_stream)

    def results(self):
        """(stats, selected seeds, windows, fragment offsets, readback hits),
        each cut to what was stored."""
        torch.cuda.synchronize(self.batch.device)
        st = np.frombuffer(self.stats.cpu().numpy().tobytes()[: ASTATS_DTYPE.itemsize], ASTATS_DTYPE)[0].copy()
        ns = min(int(st["n_selected"]), self.seed_cap)
        nw = min(int(st["n_windows"]), self.win_cap)
        nh = min(int(st["n_hits"]), self.hit_cap)
        seeds = np.frombuffer(self.seeds[: ns * ASEED_DTYPE.itemsize].cpu().numpy().tobytes(), ASEED_DTYPE).copy()
        wins = np.frombuffer(self.windows[: nw * WINDOW_DTYPE.itemsize].cpu().numpy().tobytes(), WINDOW_DTYPE).copy()
        frag = np.frombuffer(self.frag_off[: (nw * self.n_towers + 1) * 8].cpu().numpy().tobytes(), np.uint64).copy()
        hits = np.frombuffer(self.hits[: nh * HIT_DTYPE.itemsize].cpu().numpy().tobytes(), HIT_DTYPE).copy()
        return st, seeds, wins, frag, hits
