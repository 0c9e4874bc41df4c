"""CPU oracle of the multi-tower selection -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import this module; the product never does.

What it computes (arXiv 1411.3968, "Results and perspectives": for the
eight KM3Net-It towers each tower's GPU looks for all trigger seeds of its
tower and sends them to a central CPU, which selects the muon-track
candidates and sends their times back, so that every tower ships its window
of data around them to the Event Manager).  The paper names the steps but
not the central selection rule; the reading taken here applies the
paper's time-space correlation across towers:

  seeds      the triggers of each tower's slice (``oracle.run``), tower
             by tower.
  candidate  seed s of tower a (PMT p_s, time t_s) is selected iff at least
             K towers, a included, hold a seed j with
             |t_j - t_s| <= min(dt_max(p_s, p_j), W), dt_max from the two
             PMTs' positions in the array's frame (the formula used inside a
             tower).  Its tower count is reported with it.
  order      selected seeds by (t, tower, position in the tower's list).
  windows    [t - h, t + h] around every selected seed, in that order,
             merged while lo_next <= hi_cur + 1; n_triggers = selected seeds
             inside, n_hits = hits of all towers inside.
  readback   for each window, for each tower, the tower's hits inside the
             window in the tower's stream order (PMT by PMT, time order
             within a PMT, as the producer's CSR holds them).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import HIT_DTYPE, WINDOW_DTYPE, dtmax

ASEED_DTYPE = np.dtype([("t", "<i8"), ("pmt", "<u2"), ("tower", "<u2"), ("n_towers", "<u4")])


@dataclass
class ArrayResult:
    seeds: np.ndarray       # ASEED_DTYPE, selected seeds in (t, tower, position) order
    windows: np.ndarray     # WINDOW_DTYPE
    frag_off: np.ndarray    # (n_windows * n_towers + 1,) offsets of (window, tower) fragments
    hits: np.ndarray        # HIT_DTYPE, the readback, fragment after fragment


def select(tower_xyz, params: dict, min_towers: int, corr_window_ns: int, win_half_ns: int,
           tower_seeds, tower_streams) -> ArrayResult:
    """tower_xyz[b]: (P_b, 3) PMT positions of tower b in the array frame;
    tower_seeds[b]: the tower's triggers (SEED_DTYPE, time order);
    tower_streams[b]: (hits, pmt_off), the tower's hits grouped by PMT."""
    n_t = len(tower_xyz)
    base = np.concatenate([[0], np.cumsum([len(x) for x in tower_xyz])]).astype(np.int64)
    dt = dtmax(np.concatenate(tower_xyz).astype(np.int32), params)     # exact, array frame
    W = int(corr_window_ns)

    picked = []
    for a in range(n_t):
        Sa = tower_seeds[a]
        for pos in range(len(Sa)):
            ts, ps = int(Sa["t"][pos]), int(Sa["pmt"][pos])
            towers = 0
            for b in range(n_t):
                Sb = tower_seeds[b]
                lo = int(np.searchsorted(Sb["t"], ts - W, "left"))
                hi = int(np.searchsorted(Sb["t"], ts + W, "right"))
                for j in range(lo, hi):
                    lim = min(int(dt[base[a] + ps, base[b] + int(Sb["pmt"][j])]), W)
                    if abs(int(Sb["t"][j]) - ts) <= lim:
                        towers += 1
                        break
            if towers >= min_towers:
                picked.append((ts, a, pos, ps, towers))
    picked.sort()
    seeds = np.zeros(len(picked), ASEED_DTYPE)
    for i, (ts, a, _, ps, k) in enumerate(picked):
        seeds[i] = (ts, ps, a, k)

    h = int(win_half_ns)
    wins = []
    for ts in seeds["t"].tolist():
        lo, hi = ts - h, ts + h
        if wins and lo <= wins[-1][1] + 1:
            wins[-1][1] = max(wins[-1][1], hi)
            wins[-1][3] += 1
        else:
            wins.append([lo, hi, 0, 1])
    n_w = len(wins)
    wlo = np.array([w[0] for w in wins], np.int64)
    whi = np.array([w[1] for w in wins], np.int64)

    # each tower's hits inside a window, tagged (window, tower, CSR position)
    parts = []
    for b in range(n_t):
        hits, _ = tower_streams[b]
        t = hits["t"].astype(np.int64)
        w = np.searchsorted(wlo, t, "right") - 1
        inside = (w >= 0) & (t <= whi[np.maximum(w, 0)]) if n_w else np.zeros(len(t), bool)
        idx = np.nonzero(inside)[0]
        parts.append((w[idx], np.full(len(idx), b), idx, hits[idx]))
    if parts:
        wi = np.concatenate([p[0] for p in parts])
        tb = np.concatenate([p[1] for p in parts])
        pos = np.concatenate([p[2] for p in parts])
        hh = np.concatenate([p[3] for p in parts]) if len(wi) else np.zeros(0, HIT_DTYPE)
    else:
        wi = tb = pos = np.zeros(0, np.int64)
        hh = np.zeros(0, HIT_DTYPE)
    order = np.lexsort((pos, tb, wi))
    out_hits = np.ascontiguousarray(hh[order], HIT_DTYPE)
    frag = np.zeros(n_w * n_t + 1, np.uint64)
    if len(wi):
        np.add.at(frag, (wi * n_t + tb + 1).astype(np.int64), 1)
    frag = np.cumsum(frag).astype(np.uint64)
    windows = np.zeros(n_w, WINDOW_DTYPE)
    for k, w in enumerate(wins):
        windows[k] = (w[0], w[1], int(frag[(k + 1) * n_t] - frag[k * n_t]), w[3])
    return ArrayResult(seeds, windows, frag, out_hits)
