"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): every rank
solves its own replica (its own seed), timings are combined by an element-wise
maximum over ranks, and the job rate counts all ranks' updates."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # per-rank timings: the slowest rank sets every entry
        t = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 0.25 * (rank + 1)], torch.device("cpu"))
        # replicas: each rank's box comes from its own seed
        chi = synth.random_box(6, 5, 4, seed=rank)["chi"]
        allc = [torch.zeros(chi.size, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(allc, torch.from_numpy(chi.ravel().copy()))
        distinct = not torch.equal(allc[0], allc[1])
        out[rank] = (t, distinct)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_timings_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for rank in (0, 1):
        t, distinct = res[rank]
        assert t == [2.0, 5.0, 0.5]
        assert distinct


def test_job_throughput_counts_every_replica():
    import bench
    assert bench.job_throughput(1000, 4, 0.5) == 8000.0
    assert np.isclose(bench.job_throughput(7, 1, 2.0), 3.5)
