"""Biquadratic (9-point) interpolation at M and P on the GPU (Sec. 3.1;
porta_set_interpolation(2), the general sweep) against the oracle's
biquadratic sweep: J^K_Q and Lambda-bar* of a formal solution in several launch
shapes (strips of 2 to 10 rows, ragged, the stencil reaching the previous and
next CTAs' rows), and emergent Stokes vectors. Tolerances as the bilinear
parity tests (the same arithmetic with more corners): FP64 1e-10, FP32 1e-5.
The atmospheres are smooth: on rough ones (the benchmark's random boxes) the
9-point interpolant of the opacity can turn negative, in the oracle as on the
GPU, and the option is for smooth atmospheres."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import initial_rho, make_ctx, polarized_case

pytestmark = pytest.mark.gpu


def _check(jg, lg, jo, lo, tol):
    s = np.abs(jo[..., :1])
    assert np.max(np.abs(jg - jo) / s) < tol
    assert np.max(np.abs(lg - lo) / np.abs(lo)) < tol


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
@pytest.mark.parametrize("cluster", [1, 2, 3, 5])
def test_biquadratic_formal_solution_matches_oracle_polarized(prec, tol, cluster):
    atm = synth.random_box(9, 11, 10, seed=15, sigma_lnchi=0.05, sigma_v=0.1)
    rho = initial_rho(atm, 1, seed=16)
    quad = (2, 4, 7)
    ctx = make_ctx(atm, 1, *quad, prec, cluster=cluster, rho=rho)
    ctx.set_interpolation(2)
    ctx.formal_solve()
    assert ctx.launch_info()["cluster"] == cluster
    jg, lg = ctx.accumulate_jkq()
    jo, lo = oracle.formal_solve(oracle.Problem(atm, 1, *quad, interp=2), rho)
    _check(jg, lg, jo, lo, tol)
    # and it differs from the bilinear solution (the stencils are not the same)
    jb, _ = oracle.formal_solve(oracle.Problem(atm, 1, *quad, interp=1), rho)
    assert np.max(np.abs(jb - jo) / np.abs(jo[..., :1])) > 100 * tol
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_biquadratic_unpolarized_and_emergent(prec, tol):
    atm = synth.plane_parallel_box(8, 12, 14, modulation=0.2)
    atm["vel"] = 0.3 * np.sin(2 * np.pi * np.arange(8) / 8.0)[None, None, :] * np.ones((14, 12, 8))
    # a smooth, horizontally varying source function
    xx, yy = np.meshgrid(np.arange(8) / 8.0, np.arange(12) / 12.0)
    rho = initial_rho(atm, 0)
    rho[..., 0] *= (1.0 + 0.3 * np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * yy))[None, :, :]
    rho[..., 0] *= np.linspace(0.5, 1.5, 14)[:, None, None]
    ctx = make_ctx(atm, 0, 2, 4, 5, prec, rho=rho)
    ctx.set_interpolation(2)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    p = oracle.Problem(atm, 0, 2, 4, 5, interp=2)
    jo, lo = oracle.formal_solve(p, rho)
    _check(jg, lg, jo, lo, tol)
    mu = np.array([1.0, 0.31, 0.7])
    chi = np.array([0.0, 2.2, 4.0])
    eg = ctx.emergent_stokes(mu, chi)
    eo = oracle.emergent(p, rho, mu, chi)
    assert np.max(np.abs(eg - eo) / np.abs(eo[..., :1])) < tol
    ctx.close()


def test_interpolation_option_errors():
    atm = polarized_case(6, 6, 8, seed=18)
    ctx = make_ctx(atm, 1, 1, 2, 3, P.PORTA_FP64)
    with pytest.raises(P.PortaError) as e:
        ctx.set_interpolation(3)
    assert e.value.code == P.PORTA_EINVAL
    ctx.set_interpolation(2)
    with pytest.raises(P.PortaError) as e:
        ctx.emergent_vjp(np.array([1.0]), np.array([0.0]), np.ones((1, 3, 6, 6, 4)))
    assert e.value.code == P.PORTA_EINVAL
    ctx.set_interpolation(1)
    ctx.formal_solve()
    ctx.close()
