"""Batched problems: many boxes of uneven size in one persistent launch per
formal solution (porta_batch_create), against the oracle box by box."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import initial_rho

pytestmark = pytest.mark.gpu


def _boxes():
    # uneven sizes: x and y extents, depths, one box narrower than the cluster sizes
    dims = [(8, 8, 16), (16, 16, 10), (24, 24, 7), (5, 12, 9), (12, 5, 6), (3, 3, 20)]
    return [synth.random_box(nx, ny, nz, seed=[40, b]) for b, (nx, ny, nz) in enumerate(dims)]


def _rho(atms, seed):
    return [initial_rho(a, 1, seed=seed + b).reshape(-1, 6) for b, a in enumerate(atms)]


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_batch_matches_oracle_per_box(prec, tol):
    atms = _boxes()
    rhos = _rho(atms, 50)
    ctx = P.BatchContext(atms, 1, 2, 4, 9, precision=prec)
    ctx.set_atmosphere(atms)
    ctx.set_rho(np.concatenate(rhos))
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    for b, (atm, jb, lb) in enumerate(zip(atms, ctx.split(jg), ctx.split(lg))):
        p = oracle.Problem(atm, 1, 2, 4, 9)
        jo, lo = oracle.formal_solve(p, rhos[b].reshape(p.shape + (6,)))
        jo = jo.reshape(-1, 6)
        lo = lo.ravel()
        assert np.max(np.abs(jb - jo) / np.abs(jo[:, :1])) < tol, b
        assert np.max(np.abs(lb - lo) / np.abs(lo)) < tol, b


def test_batch_jacobi_step_and_launch_shapes():
    atms = _boxes()
    rhos = _rho(atms, 60)
    ref = None
    for cluster, nu in [(1, 2), (2, 4), (4, 3), (8, 9)]:
        ctx = P.BatchContext(atms, 1, 2, 4, 9, precision=P.PORTA_FP64, cluster=cluster, nu_group=nu)
        ctx.set_atmosphere(atms)
        ctx.set_rho(np.concatenate(rhos))
        ctx.formal_solve()
        ctx.accumulate_jkq(want=False)
        mc = ctx.see_update()
        rho = ctx.get_rho(np.zeros((ctx.nvox, 6)))
        if ref is None:
            ref = (rho, mc)
            # oracle Jacobi step box by box
            mco = 0.0
            for b, atm in enumerate(atms):
                p = oracle.Problem(atm, 1, 2, 4, 9)
                r0 = rhos[b].reshape(p.shape + (6,))
                jo, lo = oracle.formal_solve(p, r0)
                ro, m = oracle.see_update(p, jo, lo, r0)
                mco = max(mco, m)
                rb = ctx.split(rho)[b]
                assert np.max(np.abs(rb - ro.reshape(-1, 6)) / np.abs(ro.reshape(-1, 6)[:, :1])) < 1e-10
            assert abs(mc - mco) < 1e-9 * mco
        else:
            assert np.max(np.abs(rho - ref[0]) / np.abs(ref[0][:, :1])) < 1e-12
        ctx.close()


def test_batched_256_box_configuration_sampled():
    """The 256-box batch (Nx = Ny in {8..48}, Nz in 16..64, 80 rays, 21 frequencies,
    FP32 sweeps): one formal solution; three boxes checked against the oracle and
    invariants (J^0_0 > 0, 0 <= Lambda-bar* < 1) on all voxels."""
    atms = synth.batched_boxes(256, seed=0)
    ctx = P.BatchContext(atms, 1, 4, 10, 21, precision=P.PORTA_FP32)
    ctx.set_atmosphere(atms)
    rhos = [initial_rho(a, 1).reshape(-1, 6) for a in atms]
    ctx.set_rho(np.concatenate(rhos))
    ctx.autotune()
    ctx.set_rho(np.concatenate(rhos))
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    assert np.all(jg[:, 0] > 0) and np.all(lg >= 0) and np.all(lg < 1)
    sizes = [a["nx"] * a["ny"] * a["nz"] for a in atms]
    for b in [int(np.argmin(sizes)), 17, 101]:
        atm = atms[b]
        p = oracle.Problem(atm, 1, 4, 10, 21)
        jo, lo = oracle.formal_solve(p, rhos[b].reshape(p.shape + (6,)))
        jb, lb = ctx.split(jg)[b], ctx.split(lg)[b]
        assert np.max(np.abs(jb - jo.reshape(-1, 6)) / np.abs(jo.reshape(-1, 6)[:, :1])) < 1e-5, b
        assert np.max(np.abs(lb - lo.ravel()) / np.abs(lo.ravel())) < 1e-5, b
