"""Frequency bands of a formal solution on the GPU (the band split of Sec. 4.3
that paper_1307_4217_gb300.shard runs over ranks), emulated on one GPU with
one context per band: the bands' partial sums (porta_get_partial), added
element-wise, loaded into a context (porta_set_partial), give the J^K_Q and
Lambda-bar* of the whole frequency grid and the same update.

FP64: doubles, 1e-12 of J^0_0. FP32: int64 fixed-point sums, exact to add; a
band's passes group its frequencies differently from the whole grid's, so the
FP32 rounding of the per-pass sums differs: 1e-6 relative (the FP32 form's
parity tolerance is 1e-5). The update divides a change of J by
1 - (1 - eps) Lambda-bar* (down to ~eps = 1e-3 in thick layers), so the updated
unknowns agree to 1e-9 (FP64) and 1e-4 (FP32, the converged-rho tolerance)."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
from gpu_util import initial_rho, make_ctx, polarized_case
from paper_1307_4217_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol,rtol", [(P.PORTA_FP64, 1e-12, 1e-9), (P.PORTA_FP32, 1e-6, 1e-4)])
@pytest.mark.parametrize("world", [2, 3])
def test_band_partials_add_up_to_the_whole_grid(prec, tol, rtol, world):
    atm = polarized_case(12, 10, 16, seed=41)
    rho = initial_rho(atm, 1, seed=42)
    quad = (3, 8, 21)
    full = make_ctx(atm, 1, *quad, prec, rho=rho)
    full.formal_solve()
    jf, lf = full.accumulate_jkq()
    total = None
    ctxs = []
    for r, band in enumerate(shard.freq_bands(quad[2], world)):
        c = make_ctx(atm, 1, *quad, prec, rho=rho)
        c.set_freq_range(*band)
        c.formal_solve()
        part = c.get_partial()
        total = part.copy() if total is None else total + part
        ctxs.append(c)
    # the summed partials become rank 0's J^K_Q; the update follows as on one rank
    c0 = ctxs[0]
    c0.set_partial(total)
    jb, lb = c0.accumulate_jkq()
    scale = np.abs(jf[..., :1])
    assert np.max(np.abs(jb - jf) / scale) < tol
    assert np.max(np.abs(lb - lf) / np.abs(lf)) < tol
    ch_b = c0.see_update()
    ch_f = full.see_update()
    rb, rf = c0.get_rho(), full.get_rho()
    assert np.max(np.abs(rb - rf) / np.abs(rf[..., :1])) < rtol
    assert abs(ch_b - ch_f) <= rtol * max(ch_f, 1e-30) + 1e-14
    # and the whole grid matches the oracle
    jo, lo = oracle.formal_solve(oracle.Problem(atm, 1, *quad), rho)
    assert np.max(np.abs(jb - jo) / np.abs(jo[..., :1])) < (1e-10 if prec == P.PORTA_FP64 else 1e-5)
    for c in ctxs + [full]:
        c.close()


def test_band_bounds_are_checked():
    atm = polarized_case(6, 5, 8, seed=43)
    c = make_ctx(atm, 1, 2, 4, 7, P.PORTA_FP32)
    for j0, j1 in [(-1, 3), (3, 3), (2, 8), (5, 4)]:
        with pytest.raises(P.PortaError):
            c.set_freq_range(j0, j1)
    c.set_freq_range(2, 5)
    with pytest.raises(P.PortaError):
        c.probe_ray(0)                       # probes need the whole grid
    c.set_freq_range(0, 0)
    c.probe_ray(0)
    c.close()
