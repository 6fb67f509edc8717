"""Multi-rank host logic on CPU (gloo, world size 2): queries are sharded across
ranks with no data-path collective; only the timing max and the edge sum are
reduced. Each rank runs the CPU oracle on its shard, and the union of the
shards equals the single-rank work."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import sys
    from pathlib import Path

    root = Path(__file__).resolve().parent.parent
    sys.path.insert(0, str(root))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1607_05707_gb300 import inputs

    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = inputs.rmat(11, 8, seed=3, weights=True)
    srcs = list(inputs.sources(g, 7, seed=4))
    mine = bench.shard(srcs, world, rank)
    edges = 0
    for s in mine:
        edges += bench.reached_stats(g, oracle.bfs(g.n, g.row_ptr, g.col, [s]))[1]
    t_local = float(rank + 1)  # stand-in per-rank time
    t_max = bench.max_over_ranks(t_local, world)
    e_all = bench.sum_over_ranks(edges, world)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([len(mine), edges, t_max, e_all], dtype=np.float64))
    np.save(os.path.join(out_dir, f"s{rank}.npy"), np.array(mine, dtype=np.uint32))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_queries_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    r = [np.load(tmp_path / f"r{i}.npy") for i in range(world)]
    shards = [np.load(tmp_path / f"s{i}.npy") for i in range(world)]
    # every rank saw the same reductions: max time and total edges
    assert r[0][2] == r[1][2] == 2.0
    assert r[0][3] == r[1][3] == r[0][1] + r[1][1]
    # the shards partition the query list
    import bench
    import oracle
    from paper_1607_05707_gb300 import inputs

    g = inputs.rmat(11, 8, seed=3, weights=True)
    srcs = list(inputs.sources(g, 7, seed=4))
    assert sorted(np.concatenate(shards).tolist()) == sorted(int(s) for s in srcs)
    total = sum(bench.reached_stats(g, oracle.bfs(g.n, g.row_ptr, g.col, [s]))[1] for s in srcs)
    assert r[0][3] == total
