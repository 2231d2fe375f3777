"""Non-linear multigrid V-cycle on the GPU (porta_mg_setup / porta_mg_vcycle)
against the oracle's V-cycle (oracle/mg.py) from the same starting point, and
its convergence to the fine-grid solution.

Tolerances: FP64, one V-cycle involves ~20 formal solutions on three grids
whose J^K_Q agree with the oracle to ~1e-13; the Jacobi steps divide by
1 - (1-eps) Lambda* >= ~eps, so the unknowns agree to 1e-9. FP32: J^K_Q
carries ~1e-6 relative error, amplified by the same divisor (eps = 1e-2 here)
and accumulated over the smoothing sweeps: 1e-4 relative on S^0_0 and 1e-5
on S^2_Q / S^0_0 (the precision form's stated tolerance for rho).
"""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import initial_rho, make_ctx
from oracle import mg

pytestmark = pytest.mark.gpu

QUAD = (2, 4, 3)


def _atm(nx, ny, nz, pol, seed=5):
    if pol:
        a = synth.random_box(nx, ny, nz, seed=seed, tau_top=1e-2, tau_bot=1e2)
    else:
        a = synth.plane_parallel_box(nx, ny, nz, modulation=0.3, tau_top=1e-2, tau_bot=1e2)
        a["vel"] = 0.5 * np.random.default_rng(seed).normal(size=a["chi"].shape)
    a["eps"] = np.full_like(a["eps"], 1e-2)
    return a


def _cmp_rho(g, o, tol_rel, tol_pol):
    assert np.max(np.abs(g[..., 0] - o[..., 0]) / np.abs(o[..., 0])) < tol_rel
    if o.shape[-1] > 1:
        assert np.max(np.abs(g[..., 1:] / g[..., :1] - o[..., 1:] / o[..., :1])) < tol_pol


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
@pytest.mark.parametrize("pol,nz", [(False, 17), (True, 16), (True, 17)])
def test_vcycle_matches_oracle(prec, pol, nz):
    atm = _atm(8, 8, nz, pol)
    model = 1 if pol else 0
    rho0 = initial_rho(atm, model)
    ctx = make_ctx(atm, model, *QUAD, prec, rho=rho0)
    ctx.mg_setup(3)
    nc = mg.coarse_nz(nz)
    assert ctx.mg_levels() == [(8, 8, nz), (4, 4, nc), (2, 2, mg.coarse_nz(nc))]
    levels = mg.hierarchy(atm, model, QUAD, 3)
    ro = rho0.copy()
    for cycle in range(2):
        mc = ctx.mg_vcycle(2, 4, 8)
        ro_prev = ro
        ro = mg.vcycle(levels, ro, npre=2, npost=4, ncoarse=8)
        rg = ctx.get_rho()
        if prec == P.PORTA_FP64:
            _cmp_rho(rg, ro, 1e-9, 1e-10)
        else:
            _cmp_rho(rg, ro, 1e-4, 1e-5)
        # the reported change is the cycle's maximum relative change of S^0_0 and S^2/S^0_0
        ch = np.max(np.abs(ro[..., 0] - ro_prev[..., 0]) / np.abs(ro_prev[..., 0]))
        if pol:
            ch = max(ch, np.max(np.abs(ro[..., 1:] / ro[..., :1] - ro_prev[..., 1:] / ro_prev[..., :1])))
        assert abs(mc - ch) <= (1e-8 if prec == P.PORTA_FP64 else 1e-3) * max(ch, 1e-12)


def test_vcycles_reach_the_jacobi_fixed_point():
    torch = pytest.importorskip("torch")
    atm = _atm(16, 16, 33, True, seed=9)
    rho0 = initial_rho(atm, 1)
    jac = make_ctx(atm, 1, *QUAD, P.PORTA_FP64, rho=rho0)
    jac.set_stream(torch.cuda.Stream())
    for _ in range(40):
        mcj = jac.run_iterations(25)
        if mcj < 1e-13:
            break
    assert mcj < 1e-12
    ref = jac.get_rho()
    ctx = make_ctx(atm, 1, *QUAD, P.PORTA_FP64, rho=rho0)
    ctx.mg_setup(3)
    changes = [ctx.mg_vcycle(2, 4, 8) for _ in range(14)]
    assert changes[-1] < 1e-9
    assert changes[4] < 1e-2 * changes[0]
    _cmp_rho(ctx.get_rho(), ref, 1e-8, 1e-9)


def test_mg_setup_and_vcycle_errors():
    atm = _atm(6, 8, 9, False)
    ctx = make_ctx(atm, 0, *QUAD, P.PORTA_FP64)
    with pytest.raises(P.PortaError) as e:
        ctx.mg_vcycle()
    assert e.value.code == P.PORTA_ESTATE
    with pytest.raises(P.PortaError) as e:
        ctx.mg_setup(3)                     # 6 is not divisible by 4
    assert e.value.code == P.PORTA_EINVAL
    ctx.mg_setup(2)
    assert ctx.mg_levels() == [(6, 8, 9), (3, 4, 5)]
    ctx.mg_vcycle(1, 1, 2)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
@pytest.mark.parametrize("pol,nz", [(False, 17), (True, 16)])
def test_cubic_vcycle_and_nested_cycle_match_oracle(prec, pol, nz):
    """Tri-cubic-centered prolongation (Sec. 5.2) and the nested method (Sec. 5.1)
    against oracle/mg.py; same tolerances as the tri-linear cycle."""
    atm = _atm(16, 16, nz, pol)
    model = 1 if pol else 0
    rho0 = initial_rho(atm, model)
    levels = mg.hierarchy(atm, model, QUAD, 3)
    tol = (1e-9, 1e-10) if prec == P.PORTA_FP64 else (1e-4, 1e-5)
    ctx = make_ctx(atm, model, *QUAD, prec, rho=rho0)
    ctx.mg_setup(3)
    ctx.mg_set_prolongation(3)
    ro = rho0.copy()
    for _ in range(2):
        ctx.mg_vcycle(2, 4, 8)
        ro = mg.vcycle(levels, ro, npre=2, npost=4, ncoarse=8, order=3)
        _cmp_rho(ctx.get_rho(), ro, *tol)
    ctx.close()
    # nested: from the injection of S^0_0 = B, S^2_Q = 0 on the coarsest grid
    ctx = make_ctx(atm, model, *QUAD, prec, rho=rho0)
    ctx.mg_setup(3)
    ctx.mg_set_prolongation(3)
    ctx.mg_nested(1, 2, 4, 8)
    rc0 = initial_rho(levels[-1].atm, model)
    rn = mg.nested(levels, rc0, ncycles=1, npre=2, npost=4, ncoarse=8, order=3)
    _cmp_rho(ctx.get_rho(), rn, *tol)
    ctx.close()


def test_mg_prolongation_option_errors():
    atm = _atm(8, 8, 17, False)
    ctx = make_ctx(atm, 0, *QUAD, P.PORTA_FP64, rho=initial_rho(atm, 0))
    with pytest.raises(P.PortaError) as e:
        ctx.mg_set_prolongation(3)
    assert e.value.code == P.PORTA_ESTATE
    ctx.mg_setup(3)                          # 8 -> 4 -> 2: too few coarse nodes for the cubic
    with pytest.raises(P.PortaError) as e:
        ctx.mg_set_prolongation(3)
    assert e.value.code == P.PORTA_EINVAL
    with pytest.raises(P.PortaError) as e:
        ctx.mg_set_prolongation(2)
    assert e.value.code == P.PORTA_EINVAL
    with pytest.raises(P.PortaError) as e:
        ctx.mg_nested(0)
    assert e.value.code == P.PORTA_EINVAL
    ctx.mg_set_prolongation(1)
    ctx.mg_nested(1, 1, 1, 2)
