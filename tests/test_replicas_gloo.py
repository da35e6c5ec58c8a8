"""Multi-process (gloo, world size 2, CPU) checks of the replica path: each
rank owns a disjoint slice of the environments; results must equal the
single-process run bit for bit (environments do not couple, Sec. IV-B.3),
and the benchmark's aggregation takes the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2604_17513_gb300 import scenes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = scenes.cloth_gripper(n_envs=4, n_side=8, side=0.15, steps=4)
    lo, hi = bench.shard(sc.n_envs, rank, world)
    res = {}
    for e in range(lo, hi):
        st = oracle.rollout(sc, e, 3)
        res[e] = st.q.copy()
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    ms = 10.0 + rank                     # rank 1 is the slow one
    value, ms_max = bench.aggregate(ms, hi - lo, world, torch.device("cpu"))
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        np.save(out, np.stack([merged[e] for e in range(sc.n_envs)]))
        with open(out + ".agg", "w") as f:
            f.write(f"{value} {ms_max}")
    dist.destroy_process_group()


def test_two_rank_shards_match_single_process(tmp_path):
    import oracle
    from paper_2604_17513_gb300 import scenes
    oracle.build()
    out = str(tmp_path / "q.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    q2 = np.load(out)
    sc = scenes.cloth_gripper(n_envs=4, n_side=8, side=0.15, steps=4)
    for e in range(4):
        st = oracle.rollout(sc, e, 3)
        assert np.array_equal(st.q, q2[e])
    value, ms_max = map(float, open(out + ".agg").read().split())
    assert ms_max == 11.0
    assert abs(value - 4 / 11.0 * 1e3) < 1e-9
