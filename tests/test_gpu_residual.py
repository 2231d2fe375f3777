"""The residual of A(x) = f (porta_residual; the multigrid section's Eq. 30 at
the current unknowns) against the oracle's: a formal solution, A(S) from the
oracle's operator (or_see_apply), f = eps B delta_K0, and the maximum over
voxels of max_c |r_c| / max_c |x_c|; and it falls under Jacobi iterations."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
from gpu_util import initial_rho, make_ctx, polarized_case, unpolarized_case

pytestmark = pytest.mark.gpu


def _oracle_residual(atm, model, quad, rho):
    p = oracle.Problem(atm, model, *quad)
    j, l = oracle.formal_solve(p, rho)
    a = oracle.see_apply(p, j, rho)
    f = np.zeros_like(rho)
    f[..., 0] = np.asarray(atm["eps"]) * np.asarray(atm["bpl"])
    r = f - a
    return float(np.max(np.max(np.abs(r), axis=-1) / np.max(np.abs(rho), axis=-1)))


@pytest.mark.parametrize("model", [0, 1])
def test_residual_matches_the_oracle_and_falls_under_jacobi(model):
    atm = unpolarized_case(8, 8, 12, seed=51) if model == 0 else polarized_case(8, 8, 12, seed=52)
    quad = (2, 4, 7)
    rho = initial_rho(atm, model, seed=53 if model else None)
    ctx = make_ctx(atm, model, *quad, P.PORTA_FP64, rho=rho)
    r0 = ctx.residual()
    want = _oracle_residual(atm, model, quad, rho)
    assert abs(r0 - want) <= 1e-9 * want, (r0, want)
    for _ in range(5):
        ctx.formal_solve()
        ctx.accumulate_jkq(want=False)
        ctx.see_update(residual=False)
    r5 = ctx.residual()
    assert r5 < 0.5 * r0, (r0, r5)
    ctx.close()
