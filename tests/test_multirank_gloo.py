"""The multi-rank path on CPU (world size 2, gloo): every rank takes its
uniform-matrix-distribution slice of the operators (Sec. 3.2), rotates it, and the
slices gathered on rank 0 equal the single-process result; the job time is the
maximum over ranks, as bench.py reports it.  The rotation of each slice is the
oracle here (no GPU on this host); the partition and gather logic are the ones the
benchmark uses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_0909_5662_gb300.partition import umd_partition
        from workloads import dense_workload
        w = dense_workload("mr", 77, 4, 12, 10, 7)       # same seeded inputs on every rank
        lo, hi = umd_partition(w.K, world, rank)
        mine = oracle.rotate_dense(w.U, w.O[lo:hi], w.d, nthreads=1) if hi > lo else \
            np.zeros((0, w.mp, w.mp))
        # gather variable-size slices: pad to the largest slice
        cap = max(umd_partition(w.K, world, r)[1] - umd_partition(w.K, world, r)[0] for r in range(world))
        buf = torch.zeros((cap, w.mp, w.mp), dtype=torch.float64)
        buf[: hi - lo] = torch.from_numpy(mine)
        parts = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            full = []
            for r in range(world):
                a, b = umd_partition(w.K, world, r)
                full.append(parts[r][: b - a].numpy())
            got = np.concatenate(full)
            ref = oracle.rotate_dense(w.U, w.O, w.d, nthreads=1)
            np.save(result_path, np.array([np.abs(got - ref).max(), t.item(), len(got)]))
    finally:
        dist.destroy_process_group()


def test_two_rank_umd_partition_gloo(tmp_path):
    world = 2
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    err, tmax, n = np.load(out)
    assert err == 0.0          # bit-identical: the same oracle loops on the same operators
    assert tmax == 2.0         # max over ranks
    assert n == 7
