"""Pins of the family of formal solvers compared on the sigmoid benchmark
(Sec. 3.4, Fig. 5): linear and parabolic short characteristics, the quadratic
Bezier spline with the Fritsch-Butland derivative at O without (BEZIER_FB) and
with (CBEZIER) the upwind overshoot correction, and BESSER. The Fritsch-Butland
derivative is checked against scipy's PCHIP (an independent implementation of
the same weighted harmonic mean), the exactness of each method against
quadrature, the derivatives of exponential data against closed forms, and the
benchmark's convergence orders and the BESSER/parabolic relations that Sec. 3.4
states."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.interpolate import PchipInterpolator

import oracle

FAMILY = [oracle.BESSER, oracle.DELOPAR, oracle.LINEAR, oracle.BEZIER_FB, oracle.CBEZIER]


def _ref_solution(tau, S_fun, I0):
    """I on the nodes by quadrature of S(tau) e^-t over each interval."""
    ref = np.empty_like(tau)
    ref[0] = I0
    for i in range(1, len(tau)):
        h = tau[i] - tau[i - 1]
        integ = integrate.quad(lambda t: S_fun(tau[i] - t, i) * math.exp(-t), 0, h, epsabs=0, epsrel=1e-13)[0]
        ref[i] = ref[i - 1] * math.exp(-h) + integ
    return ref


def test_fritsch_butland_derivative_is_the_pchip_interior_derivative():
    rng = np.random.default_rng(11)
    for _ in range(3000):
        hM, hP = rng.uniform(0.01, 3.0, 2)
        yM, yO, yP = rng.normal(size=3) * rng.choice([1e-3, 1.0, 1e3])
        d_ref = float(PchipInterpolator([0.0, hM, hM + hP], [yM, yO, yP]).derivative()(hM))
        for m in (oracle.BEZIER_FB, oracle.CBEZIER):
            cM = oracle.control_point(yM, yO, yP, hM, hP, True, m)
            if m == oracle.CBEZIER and cM == yM and d_ref != 0.0:
                continue                           # clipped: checked below
            d = 2.0 * (yO - cM) / hM
            assert d == pytest.approx(d_ref, rel=1e-10, abs=1e-12 * max(abs(yM), abs(yO), abs(yP)) / hM)


def test_cbezier_clips_the_upwind_overshoot_of_the_fritsch_butland_estimate():
    # h_P << h_M puts the weight alpha near 1/3, so y'_O -> 3 d_M: c_M falls below y_M
    yM, yO, yP, hM, hP = 0.0, 1.0, 11.0, 1.0, 0.01
    c_fb = oracle.control_point(yM, yO, yP, hM, hP, True, oracle.BEZIER_FB)
    assert c_fb < yM
    assert oracle.control_point(yM, yO, yP, hM, hP, True, oracle.CBEZIER) == yM
    assert oracle.control_point(yM, yO, yP, hM, hP, True, oracle.BESSER) == yM    # steps 5-6
    # an extremum at O: no slope, c_M = y_O for both Bezier forms
    for m in (oracle.BEZIER_FB, oracle.CBEZIER):
        assert oracle.control_point(0.0, 1.0, 0.5, 0.7, 0.3, True, m) == 1.0


def test_derivative_estimates_for_exponential_data_match_closed_forms():
    """For y = exp(-2z) on a uniform grid the harmonic mean of the one-sided slopes is
    -2 y_O tanh(h)/h and the parabolic derivative (Eq. 6) is -y_O sinh(2h)/h."""
    for h in [0.01, 0.1, 0.5, 1.3]:
        yM, yO, yP = math.exp(2 * h), 1.0, math.exp(-2 * h)
        d_fb = 2.0 * (yO - oracle.control_point(yM, yO, yP, h, h, True, oracle.BEZIER_FB)) / h
        d_pa = 2.0 * (yO - oracle.control_point(yM, yO, yP, h, h, True, oracle.DELOPAR)) / h
        assert d_fb == pytest.approx(-2.0 * math.tanh(h) / h, rel=1e-12)
        assert d_pa == pytest.approx(-math.sinh(2 * h) / h, rel=1e-12)


def test_linear_method_is_exact_for_piecewise_linear_source():
    rng = np.random.default_rng(3)
    tau = np.concatenate([[0.0], np.cumsum(rng.uniform(0.02, 2.0, 30))])
    S = rng.uniform(0.2, 3.0, tau.size)

    def S_lin(t, i):   # linear between S[i-1] at tau[i-1] and S[i] at tau[i]
        h = tau[i] - tau[i - 1]
        return S[i - 1] + (S[i] - S[i - 1]) * (t - tau[i - 1]) / h

    ref = _ref_solution(tau, S_lin, 0.3)
    assert np.allclose(oracle.solve_1d(tau, S, 0.3, oracle.LINEAR), ref, rtol=1e-11, atol=0)


def test_bezier_fb_is_exact_for_linear_but_not_quadratic_source():
    """Sec. 3.4: the Fritsch-Butland estimate of y'_O does not reproduce second-order
    polynomials, while the parabola (DELOPAR) does."""
    tau = np.arange(0.0, 12.0, 0.5)
    lin = lambda x: 2.0 + 0.7 * x
    quad = lambda x: 1.0 + 0.3 * x + 0.05 * x * x
    ref_lin = _ref_solution(tau, lambda t, i: lin(t), 0.4)
    ref_quad = _ref_solution(tau, lambda t, i: quad(t), 0.4)
    for m in (oracle.BEZIER_FB, oracle.CBEZIER):
        assert np.allclose(oracle.solve_1d(tau, lin(tau), 0.4, m), ref_lin, rtol=1e-11, atol=0)
        err = np.max(np.abs(oracle.solve_1d(tau, quad(tau), 0.4, m)[:-1] / ref_quad[:-1] - 1))
        assert err > 1e-5
    got = oracle.solve_1d(tau, quad(tau), 0.4, oracle.DELOPAR)
    assert np.allclose(got[:-1], ref_quad[:-1], rtol=1e-11, atol=0)


def test_sigmoid_benchmark_orders_and_besser_parabolic_relations():
    """Sec. 3.4: without overshoots BESSER and the parabola give the same solution;
    on coarse grids the parabola's overshoots make it far worse; on fine grids the
    linear method converges at second order and BESSER at third."""
    E = {m: [oracle.sigmoid_error(d, m) for d in (0.04, 0.02, 0.01)] for m in FAMILY}
    assert E[oracle.LINEAR][1] / E[oracle.LINEAR][2] == pytest.approx(4.0, rel=0.05)
    assert E[oracle.BESSER][1] / E[oracle.BESSER][2] == pytest.approx(8.0, rel=0.1)
    for d in (0.5, 0.2, 0.1, 0.02):
        assert oracle.sigmoid_error(d, oracle.BESSER) == pytest.approx(oracle.sigmoid_error(d, oracle.DELOPAR),
                                                                       rel=1e-12)
    for d in (1.0, 1.5, 2.0):
        assert oracle.sigmoid_error(d, oracle.DELOPAR) > 5.0 * oracle.sigmoid_error(d, oracle.BESSER)
    # the correction only removes overshoots: never worse than the plain Bezier form
    for d in (2.0, 1.0, 0.3, 0.05):
        for s in (0.0, 0.3 * d, 0.7 * d):
            assert oracle.sigmoid_error(d, oracle.CBEZIER, s) <= oracle.sigmoid_error(d, oracle.BEZIER_FB, s) + 1e-15


def test_sigmoid_grid_and_boundary():
    z = oracle.sigmoid_grid(0.5, 0.2)
    assert z[0] == pytest.approx(-11.8) and z[-1] <= 12.0 and 12.0 - z[-1] < 0.5
    assert np.allclose(np.diff(z), 0.5)
    assert oracle.sigmoid_exact(-12.0) == pytest.approx(2.77176e-7, rel=5e-6)
