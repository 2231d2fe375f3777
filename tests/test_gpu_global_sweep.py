"""The global-memory sweep in the plane placement (porta_set_global_sweep, faces.cu
with M and P on the neighbouring horizontal planes at any offset): the J^K_Q and
Lambda-bar* sums and the emergent profiles against the oracle's plane sweep (the
discretization of the shared-memory sweeps, Sec. 3.1 with the R3 reading), and a
box whose planes no shared-memory launch shape holds (the FP64 polarized atom on
128-wide planes), which takes it by itself. Tolerances as the bilinear parity
tests: FP64 1e-10, FP32 1e-5."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import initial_rho, make_ctx

pytestmark = pytest.mark.gpu


def _check(jg, lg, jo, lo, tol):
    s = np.abs(jo[..., :1])
    assert np.max(np.abs(jg - jo) / s) < tol
    assert np.max(np.abs(lg - lo) / np.abs(lo)) < tol


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
@pytest.mark.parametrize("model", [0, 1])
def test_global_sweep_matches_the_oracle_plane_sweep(prec, tol, model):
    atm = synth.random_box(9, 7, 10, seed=31, sigma_lnchi=0.1, sigma_v=0.3)
    rho = initial_rho(atm, model, seed=32)
    quad = (2, 4, 5)
    ctx = make_ctx(atm, model, *quad, prec, rho=rho)
    ctx.set_global_sweep(1)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    p = oracle.Problem(atm, model, *quad)
    jo, lo = oracle.formal_solve(p, rho)
    _check(jg, lg, jo, lo, tol)
    # the update from these sums is the oracle's
    ch = ctx.see_update()
    _, cho = oracle.see_update(p, jo, lo, rho)
    assert abs(ch - cho) < 10 * tol * cho
    # the shared-memory sweep of the same context gives the same sums
    ctx.set_global_sweep(0)
    ctx.set_rho(rho)
    ctx.formal_solve()
    js, ls = ctx.accumulate_jkq()
    _check(js, ls, jg, lg, tol)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_global_sweep_emergent_profiles_match_oracle(prec, tol):
    atm = synth.random_box(9, 7, 10, seed=33, sigma_lnchi=0.1, sigma_v=0.3)
    rho = initial_rho(atm, 1, seed=34)
    ctx = make_ctx(atm, 1, 2, 4, 5, prec, rho=rho)
    ctx.set_global_sweep(1)
    mu, chi = np.array([1.0, 0.5, 0.3]), np.array([0.0, 0.7, 2.1])
    eg = ctx.emergent_stokes(mu, chi)
    eo = oracle.emergent(oracle.Problem(atm, 1, 2, 4, 5), rho, mu, chi)
    assert np.max(np.abs(eg - eo)) < tol * np.max(np.abs(eo[..., 0]))
    with pytest.raises(P.PortaError):
        ctx.set_global_sweep(2)
    with pytest.raises(P.PortaError):
        ctx.set_interpolation(2)
    with pytest.raises(P.PortaError):
        ctx.emergent_vjp(mu, chi, np.ones((len(mu), 5, 7, 9, 4)))
    ctx.close()


def test_fp64_polarized_atom_on_128_wide_planes():
    """The FP64 polarized ring of a 128-wide plane does not fit shared memory: the
    context takes the global-memory sweep by itself and matches the oracle."""
    atm = synth.random_box(128, 128, 6, seed=35)
    rho = initial_rho(atm, 1, seed=36)
    quad = (1, 2, 3)
    ctx = make_ctx(atm, 1, *quad, P.PORTA_FP64, rho=rho)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    jo, lo = oracle.formal_solve(oracle.Problem(atm, 1, *quad), rho)
    _check(jg, lg, jo, lo, 1e-10)
    assert ctx.see_update() > 0
    ctx.close()
