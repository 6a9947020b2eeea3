"""Host-side logic of the multi-GPU benchmark (weak scaling, one rank per GPU, no
data-path collective), run as two gloo ranks on the CPU: the rank set-up, the
max-over-ranks timing and the sum of cells over ranks, and per-rank populations."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    from paper_1903_06479_gb300 import workloads as W
    r, w, local, pg = bench.dist_setup(world)
    t_rank = 1.0 + r  # a rank's device time
    cells = 100 + 10 * r
    out = {"rank": r, "world": w, "local": local,
           "tmax": bench.max_over_ranks(pg, t_rank), "cells": bench.sum_over_ranks(pg, cells)}
    pop = W.population(66, 2, seed=1 + r, forces="shear", noise_pN=0.5)
    out["x0"] = float(pop["x"][0, 0, 0])
    bench.barrier(pg)
    pg.destroy_process_group()
    q.put(out)


def test_two_rank_reductions_and_weak_scaling_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda d: d["rank"])
    assert [d["world"] for d in res] == [2, 2]
    assert all(d["tmax"] == 2.0 for d in res)       # slowest rank's time
    assert all(d["cells"] == 210.0 for d in res)    # whole-job cell count
    assert res[0]["x0"] != res[1]["x0"]             # each rank steps its own cells
