"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): the rank
environment, and timings combined by an element-wise maximum over ranks (the
slowest rank sets the job's time). The frequency-band split of the solver
itself is tested in test_multirank_bands.py."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp



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
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_timings():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for rank in (0, 1):
        assert res[rank] == [2.0, 5.0, 0.5]
