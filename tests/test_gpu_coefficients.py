"""The exponential-integral coefficients of the BESSER-DELO step (Eqs. 9-13)
as the sweep kernels evaluate them on the GPU, against 40-digit evaluations of
the closed forms.

FP64 bound 5e-12: just above the Table 1 crossover (t = 0.14) the closed form of
omega_M subtracts two numbers near 2 to leave ~t^3/3 = 9e-4, amplifying a few
ulps (2.2e-16 each) of rounding by ~2200. FP32 bound 1e-6: the three-regime
evaluation (series of degree 6 / 12, closed forms above t = 1.5) keeps the
truncation and cancellation errors below 6e-7."""
import mpmath
import numpy as np
import pytest

import paper_1307_4217_gb300 as P

pytestmark = pytest.mark.gpu


def _exact(t):
    mpmath.mp.dps = 40
    t = mpmath.mpf(float(t))
    e = mpmath.exp(-t)
    return [e, (1 - e * (1 + t)) / t, (e + t - 1) / t, (2 - e * (t * t + 2 * t + 2)) / t**2,
            1 - 2 * (e + t - 1) / t**2, 2 * (t - 2 + e * (t + 2)) / t**2]


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 5e-12), (P.PORTA_FP32, 1e-6)])
def test_coefficients_accuracy(prec, tol):
    t = np.geomspace(1e-7, 1e3, 2001)
    if prec == P.PORTA_FP32:
        t = t.astype(np.float32).astype(np.float64)     # the kernel sees t in FP32
    rc, out = P.porta_eval_coefficients(prec, t)
    assert rc == P.PORTA_OK
    worst = 0.0
    for i, ti in enumerate(t):
        ex = _exact(ti)
        for k in range(6):
            if ex[k] == 0 or abs(float(ex[k])) < 1e-30:
                continue
            worst = max(worst, abs(float((mpmath.mpf(out[i, k]) - ex[k]) / ex[k])))
    assert worst < tol, worst
