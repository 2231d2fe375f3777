"""The frequency-band split of a formal solution across ranks (the band
parallelization of Sec. 4.3), on CPU ranks (gloo, world size 2) with host
buffers: each rank computes its band's partial J^K_Q and Lambda-bar* (the
oracle's formal solution restricted to the band), the partial sums meet in one
all-reduce (paper_1307_4217_gb300.shard), and every rank then holds the
single-rank result to 1e-12 (FP64; the sum is the same sum regrouped) and takes
the same Jacobi update."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1307_4217_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(model):
    if model == oracle.MODEL_HANLE:
        atm = synth.random_box(6, 5, 8, seed=31)
    else:
        atm = synth.plane_parallel_box(6, 5, 8)
    p = oracle.Problem(atm, model, 2, 4, 7)
    rho = oracle.initial_rho(p, atm)
    if model == oracle.MODEL_HANLE:
        rng = np.random.default_rng(32)
        rho[..., 1:] = 0.02 * rho[..., :1] * rng.normal(size=rho.shape[:-1] + (5,))
    return atm, p, rho


def _pack(jkq, ls):
    """The FP64 partial-sum layout of porta_get_partial: J^K_Q [nvox][NJ], then Lambda-bar* [nvox]."""
    return torch.from_numpy(np.concatenate([jkq.ravel(), ls.ravel()]).copy())


def _worker(rank, world, port, model, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        atm, p, rho = _case(model)
        band = shard.freq_bands(p.n_nu, world)[rank]
        jkq, ls = oracle.formal_solve(p, rho, freq_range=band)
        buf = shard.allreduce_partial(_pack(jkq, ls))
        nj = jkq.shape[-1]
        j_all = buf[: p.nvox * nj].numpy().reshape(jkq.shape)
        l_all = buf[p.nvox * nj:].numpy().reshape(ls.shape)
        rho_new, change = oracle.see_update(p, j_all, l_all, rho)
        out[rank] = (band, j_all, l_all, rho_new, change)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("model", [oracle.MODEL_UNPOL, oracle.MODEL_HANLE])
def test_two_gloo_ranks_frequency_bands_reproduce_the_single_rank_sums(model):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), model, out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    atm, p, rho = _case(model)
    j1, l1 = oracle.formal_solve(p, rho)
    rho1, ch1 = oracle.see_update(p, j1, l1, rho)
    assert [res[r][0] for r in (0, 1)] == [(0, 4), (4, 7)]
    for r in (0, 1):
        _, j, l, rho_new, change = res[r]
        scale = np.abs(j1[..., :1])
        assert np.max(np.abs(j - j1) / scale) < 1e-12
        assert np.max(np.abs(l - l1) / np.abs(l1)) < 1e-12
        assert np.max(np.abs(rho_new - rho1) / np.abs(rho1[..., :1])) < 1e-12
        assert abs(change - ch1) <= 1e-12 * ch1
    # every rank ends with the same numbers (one all-reduce, the same update)
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][3], res[1][3])


def test_frequency_bands_partition_the_grid():
    for n_nu in (1, 7, 21, 31):
        for world in range(1, min(n_nu, 9) + 1):
            bands = shard.freq_bands(n_nu, world)
            assert bands[0][0] == 0 and bands[-1][1] == n_nu
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            sizes = [b - a for a, b in bands]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.freq_bands(4, 5)
