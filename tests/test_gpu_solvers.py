"""The GPU's family of formal solvers on the one-ray sigmoid benchmark (Sec. 3.4,
Eqs. 15-18, Fig. 5) against the oracle: E(dtau) for BESSER, the parabola, the
linear method and the two Fritsch-Butland Bezier forms, on grid spacings from 2
to 0.005 and three grid shifts. FP64: the same solver arithmetic up to rounding
order; the reference I_a of Eq. 17 cancels at the left end (at z = -12 the two
terms agree to one part in ~4e6, so each libm's I_a carries ~4e-10 relative
rounding), so E agrees to 2e-9 absolute. FP32: a rounding of ~6e-8 per step,
remembered over ~1/dtau steps per unit optical depth, so E agrees to
5e-7/dtau plus 2 % of E."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P

pytestmark = pytest.mark.gpu

PAIRS = [(P.PORTA_SC_BESSER, oracle.BESSER), (P.PORTA_SC_PARABOLIC, oracle.DELOPAR),
         (P.PORTA_SC_LINEAR, oracle.LINEAR), (P.PORTA_SC_BEZIER_FB, oracle.BEZIER_FB),
         (P.PORTA_SC_CBEZIER, oracle.CBEZIER)]
DTAU = [2.0, 1.5, 1.0, 0.7, 0.5, 0.3, 0.2, 0.1, 0.05, 0.02, 0.01, 0.005]


def _cases():
    m, d, s, ref = [], [], [], []
    for gm, om in PAIRS:
        for dt in DTAU:
            for f in (0.0, 0.37, 0.81):
                m.append(gm)
                d.append(dt)
                s.append(f * dt)
                ref.append(oracle.sigmoid_error(dt, om, f * dt))
    return np.array(m), np.array(d), np.array(s), np.array(ref)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_solver_family_matches_the_oracle_on_the_sigmoid_benchmark(prec):
    m, d, s, ref = _cases()
    rc, E = P.porta_sigmoid_error(prec, m, d, s)
    assert rc == P.PORTA_OK
    if prec == P.PORTA_FP64:
        assert np.max(np.abs(E - ref)) < 2e-9, np.max(np.abs(E - ref))
    else:
        assert np.all(np.abs(E - ref) < 5e-7 / d + 0.02 * ref), np.max(np.abs(E - ref) - 5e-7 / d - 0.02 * ref)


def test_sigmoid_error_rejects_bad_cases():
    assert P.porta_sigmoid_error(P.PORTA_FP64, [7], [0.1])[0] == P.PORTA_EINVAL
    assert P.porta_sigmoid_error(P.PORTA_FP64, [0], [0.0])[0] == P.PORTA_EINVAL
    assert P.porta_sigmoid_error(P.PORTA_FP64, [0], [0.1], [0.1])[0] == P.PORTA_EINVAL
    assert P.porta_sigmoid_error(2, [0], [0.1])[0] == P.PORTA_EINVAL
