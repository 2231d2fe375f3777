"""Frequency bands of the formal solution over the ranks of a process group.

The (ray, frequency) pairs of a formal solution are independent, and J^K_Q and
Lambda-bar* are sums over them (Eq. 1); the paper parallelizes over frequency
intervals and sums the partially integrated quantities at the end (Sec. 4.3).
Here every rank holds the whole box on its GPU, sweeps one contiguous band of
the frequency grid (porta_set_freq_range), and the ranks' partial sums meet in
one all-reduce per iteration; every rank then runs the same update (Eq. 2 with
the Jacobi step) on the same numbers. In the FP32 form the partial sums are
int64 fixed-point integers, so the all-reduce is exact and its result does not
depend on the reduction order; in the FP64 form they are doubles.

This module only partitions and moves buffers: the sweeps, the sums and the
update run in the CUDA library.
"""
import numpy as np


def freq_bands(n_nu, world):
    """Contiguous frequency bands [j0, j1) of ranks 0..world-1, covering the grid
    once; band sizes differ by at most one frequency."""
    if world < 1 or world > n_nu:
        raise ValueError(f"need 1 <= world ({world}) <= n_nu ({n_nu})")
    base, extra = divmod(n_nu, world)
    bands, j = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        bands.append((j, j + n))
        j += n
    return bands


def allreduce_partial(buf, group=None):
    """Element-wise sum over the group's ranks of a partial-sum buffer (a torch
    tensor: int64 or float64, on the device for NCCL, on the host for gloo), in place."""
    import torch.distributed as dist
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf


class BandIteration:
    """Jacobi iterations of a two-level context whose formal solution is split into
    frequency bands over `world` ranks: the rank's band is swept, the partial sums
    are all-reduced, and the update runs on every rank with the whole J^K_Q."""

    def __init__(self, ctx, rank, world, group=None, device=None):
        import torch
        self.ctx, self.rank, self.world, self.group = ctx, rank, world, group
        self.band = freq_bands(ctx.nnu, world)[rank]
        if world > 1:
            ctx.set_freq_range(*self.band)
        n = ctx.nvox * (ctx.nj + 1)
        dtype = torch.int64 if ctx.partial_dtype() == np.int64 else torch.float64
        self.buf = torch.zeros(n, dtype=dtype, device=device)

    def step(self, residual=True):
        """One iteration; returns the maximum relative change of the update (or None)."""
        c = self.ctx
        c.formal_solve()
        if self.world > 1:
            c.get_partial(self.buf)
            allreduce_partial(self.buf, self.group)
            c.set_partial(self.buf)
        else:
            c.accumulate_jkq(want=False)
        return c.see_update(residual=residual)
