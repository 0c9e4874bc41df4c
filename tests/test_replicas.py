"""Multi-rank host logic on CPU (gloo, world size 2): the replicas'
timing reductions, the partition of independent slices over ranks, and
that a sharded run gives each slice the same result as a single run (the
oracle stands in for the per-rank work; no GPU is involved)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import workload
from paper_1411_3968_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world_size, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        assert replicas.world() == (rank, world_size)
        # timing: max of the step times, sum of the hits
        mx = replicas.max_over_ranks(10.0 + rank)
        sm = replicas.sum_over_ranks(1000.0 * (rank + 1))
        # each rank triggers its share of a small contiguous run
        wl = workload.cfg_km3()
        g = wl.detectors[0]
        par = dict(workload.DEFAULT_PARAMS)
        mine = list(replicas.shard(len(wl.run_slices[0]), rank, world_size))
        t0s = [wl.run_slices[0][k] for k in mine]
        res = oracle.run(g.xyz_mm, g.floor_id, par, wl.runs[0].hits, t0s)
        replicas.barrier()
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([(mx, sm, k, len(r.triggers), len(r.windows), int(r.triggers["t"].sum()) if len(r.triggers) else 0)
                          for k, r in zip(mine, res)], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 65):
        for ws in (1, 2, 3, 8):
            got = [k for r in range(ws) for k in replicas.shard(n, r, ws)]
            assert got == list(range(n))
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_reductions_are_identity():
    assert replicas.world() == (0, 1)
    assert replicas.max_over_ranks(3.5) == 3.5 and replicas.sum_over_ranks(2.0) == 2.0


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    rows = np.concatenate([np.load(tmp_path / f"r{r}.npy") for r in range(ws)])
    assert np.all(rows[:, 0] == 11.0) and np.all(rows[:, 1] == 3000.0)
    # the sharded slices, together, equal the single-process run
    wl = workload.cfg_km3()
    g = wl.detectors[0]
    ref = oracle.run(g.xyz_mm, g.floor_id, dict(workload.DEFAULT_PARAMS), wl.runs[0].hits, wl.run_slices[0])
    assert sorted(rows[:, 2].astype(int).tolist()) == list(range(len(ref)))
    for k, nt, nw, tsum in rows[:, 2:].astype(np.int64):
        r = ref[k]
        assert nt == len(r.triggers) and nw == len(r.windows)
        assert tsum == (int(r.triggers["t"].sum()) if len(r.triggers) else 0)
