"""Pins of the oracle's BESSER formal solver (Sec. 3.2-3.4) against facts that
do not come from the oracle itself: integrals computed by quadrature, the
paper's printed numbers, Taylor series derived symbolically, and the
analytic sigmoid solution."""
import math
import os

import mpmath

import numpy as np
import pytest
from scipy import integrate

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bezier(u, yM, c, yO):
    return (1 - u) ** 2 * yM + 2 * u * (1 - u) * c + u * u * yO


@pytest.mark.parametrize("tau", [1e-3, 0.05, 0.139, 0.141, 0.179, 0.181, 0.5, 1.0, 3.7, 12.0, 60.0])
def test_omega_are_bezier_integrals(tau):
    """omega_M, omega_O, omega_C integrate the quadratic Bezier basis against e^-t
    (Eq. 7 with u = 1 - t/tau); psi'_M, psi'_O integrate the linear basis."""
    c = oracle.coeffs(tau)
    bM = integrate.quad(lambda t: _bezier(1 - t / tau, 1, 0, 0) * math.exp(-t), 0, tau, epsabs=0, epsrel=1e-13)[0]
    bO = integrate.quad(lambda t: _bezier(1 - t / tau, 0, 0, 1) * math.exp(-t), 0, tau, epsabs=0, epsrel=1e-13)[0]
    bC = integrate.quad(lambda t: _bezier(1 - t / tau, 0, 1, 0) * math.exp(-t), 0, tau, epsabs=0, epsrel=1e-13)[0]
    lM = integrate.quad(lambda t: (t / tau) * math.exp(-t), 0, tau, epsabs=0, epsrel=1e-13)[0]
    lO = integrate.quad(lambda t: (1 - t / tau) * math.exp(-t), 0, tau, epsabs=0, epsrel=1e-13)[0]
    assert c[0] == pytest.approx(math.exp(-tau), rel=1e-15)
    for got, want in [(c[1], lM), (c[2], lO), (c[3], bM), (c[4], bO), (c[5], bC)]:
        assert got == pytest.approx(want, rel=2e-12, abs=1e-300)


def test_coefficient_identities_and_lambda_range():
    mpmath.mp.dps = 40
    """w_M + w_O + w_C = psi'_M + psi'_O = 1 - e^-tau, and Lambda* = w_O + w_C in [0, 1) (Eq. 14)."""
    for tau in np.geomspace(1e-8, 1e4, 400):
        c = oracle.coeffs(tau)
        one_m_e = -math.expm1(-tau)
        assert c[3] + c[4] + c[5] == pytest.approx(one_m_e, rel=1e-12)
        assert c[1] + c[2] == pytest.approx(one_m_e, rel=1e-12)
        lam = c[4] + c[5]
        assert 0.0 <= lam < 1.0
        # Eq. 14 closed form, evaluated with 40 significant digits
        t = mpmath.mpf(tau)
        assert lam == pytest.approx(float(1 + 2 * (mpmath.exp(-t) * (1 + t) - 1) / t**2), rel=1e-11)


def test_table1_is_taylor_series_of_closed_forms():
    """The printed Table 1 polynomials are the Taylor series of Eqs. 11-13 to t^8,
    and the oracle's coefficients agree with them below the printed thresholds."""
    sp = pytest.importorskip("sympy")
    t = sp.symbols("t")
    e = sp.exp(-t)
    closed = {
        "omega_M": (2 - e * (t**2 + 2 * t + 2)) / t**2,
        "omega_O": 1 - 2 * (e + t - 1) / t**2,
        "omega_C": 2 * (t - 2 + e * (t + 2)) / t**2,
    }
    idx = {"omega_M": 3, "omega_O": 4, "omega_C": 5}
    for line in open(os.path.join(GOLDEN, "table1_series.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, rest = line.split(None, 1)
        num, rest = rest.split("/")
        den, thr = rest.split()
        num = [int(v) for v in num.split()]
        den = int(den)
        ser = sp.series(closed[name], t, 0, 9).removeO()
        for n, a in enumerate(num, start=1):
            assert sp.Rational(a, den) == ser.coeff(t, n), (name, n)
        # oracle below the threshold follows the printed polynomial
        for tv in np.linspace(1e-4, float(thr) * 0.999, 7):
            poly = sum(a * tv**n for n, a in enumerate(num, start=1)) / den
            assert oracle.coeffs(tv)[idx[name]] == pytest.approx(poly, rel=1e-14)


def _sigmoid(a, d, z):
    return 1.0 / (1.0 + np.exp(-a * (z - d)))


def _Ia(z):
    return np.exp(15 - z) / (np.exp(20) - 1) * (np.exp(10) * np.arctan(np.exp(z - 5)) - np.arctan(np.exp(z + 5)))


def test_sigmoid_analytic_solution_and_printed_boundary():
    """Eq. 17 solves dI/dz = S - I with S from Eq. 15; its value at z = -12 is the printed 2.77176e-7."""
    val, tol = [float(v) for v in open(os.path.join(GOLDEN, "sigmoid_boundary.txt")).read().split("\n")[-2].split()]
    assert _Ia(-12.0) == pytest.approx(val, rel=tol)
    mpmath.mp.dps = 50

    def Ia(z):
        return mpmath.exp(15 - z) / (mpmath.exp(20) - 1) * (
            mpmath.exp(10) * mpmath.atan(mpmath.exp(z - 5)) - mpmath.atan(mpmath.exp(z + 5)))

    def S(z):
        return 1 / (1 + mpmath.exp(-2 * (z + 5))) / (1 + mpmath.exp(2 * (z - 5)))

    for zf in np.linspace(-12, 12, 49):
        z = mpmath.mpf(zf)
        dI = mpmath.diff(Ia, z)
        assert abs((dI - (S(z) - Ia(z))) / Ia(z)) < 1e-30


def test_sigmoid_error_decreases_with_grid_spacing():
    """Sec. 3.4: the maximum true error E(dtau) of BESSER falls as the grid is refined."""
    errs = []
    for n in [25, 49, 97, 193, 385, 769]:
        z = np.linspace(-12, 12, n)
        S = _sigmoid(2, -5, z) * _sigmoid(-2, 5, z)
        I = oracle.solve_1d(z, S, _Ia(-12.0))
        errs.append(np.max(np.abs((I - _Ia(z)) / _Ia(z))))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3
    # second-order convergence on fine grids
    assert errs[-2] / errs[-1] > 3.0


@pytest.mark.parametrize("method", [oracle.BESSER, oracle.DELOPAR])
def test_linear_and_quadratic_source_are_exact(method):
    """A parabola through M, O, P is reproduced exactly (step 4 footnote), so a
    linear or monotone quadratic S(tau) gives the exact formal solution."""
    rng = np.random.default_rng(1)
    tau = np.cumsum(rng.uniform(0.05, 1.5, 40))
    tau -= tau[0]
    for S_fun, I_exact in [
        (lambda x: 2.0 + 0.7 * x, lambda x: None),
        (lambda x: 1.0 + 0.3 * x + 0.02 * x * x, lambda x: None),
    ]:
        S = S_fun(tau)
        I0 = 0.4
        I = oracle.solve_1d(tau, S, I0, method)
        ref = np.empty_like(tau)
        ref[0] = I0
        for i in range(1, len(tau)):
            h = tau[i] - tau[i - 1]
            integ = integrate.quad(lambda t: S_fun(tau[i] - t) * math.exp(-t), 0, h, epsabs=0, epsrel=1e-13)[0]
            ref[i] = ref[i - 1] * math.exp(-h) + integ
        # the last interval is linear (no downwind point): exact only for linear S
        n_chk = len(tau) if S_fun(1.0) - S_fun(0.0) == S_fun(2.0) - S_fun(1.0) else len(tau) - 1
        assert np.allclose(I[:n_chk], ref[:n_chk], rtol=1e-11, atol=0)


def _spline_samples(yM, yO, yP, hM, hP, cM, cP):
    u = np.linspace(0, 1, 201)
    left = _bezier(u, yM, cM, yO)
    right = _bezier(u, yO, cP, yP)
    return left, right


def test_besser_monotone_and_single_extremum():
    """Sec. 3.2 conditions: (1) monotone data give a monotone interpolant on [M, P];
    (2) otherwise the only extremum is at O (c_M = y_O)."""
    rng = np.random.default_rng(7)
    for _ in range(4000):
        yM, yO, yP = rng.normal(size=3) * rng.choice([1e-3, 1.0, 1e3])
        hM, hP = np.exp(rng.uniform(-4, 3, 2))
        cM = oracle.control_point(yM, yO, yP, hM, hP)
        dM, dP = (yO - yM) / hM, (yP - yO) / hP
        if dM * dP <= 0:
            assert cM == yO
            continue
        lo, hi = min(yM, yO), max(yM, yO)
        assert lo <= cM <= hi
        left = _bezier(np.linspace(0, 1, 101), yM, cM, yO)
        d = np.diff(left)
        assert np.all(d * np.sign(yO - yM) >= -1e-12 * max(abs(yM), abs(yO), 1))


def test_besser_continuous_derivative_and_parabolic_limit():
    """(3) When neither interval overshoots, BESSER is the parabola through M, O, P
    (= DELOPAR); when only OP overshoots, c_P is clipped and c_M moved so that the
    derivative at O stays continuous (steps 7-9)."""
    rng = np.random.default_rng(3)
    n_clip = 0
    for _ in range(4000):
        hM, hP = np.exp(rng.uniform(-3, 2, 2))
        yM, yO = sorted(rng.normal(size=2))
        yP = yO + abs(rng.normal()) * rng.choice([0.01, 1.0])
        cM = oracle.control_point(yM, yO, yP, hM, hP)
        cD = oracle.control_point(yM, yO, yP, hM, hP, method=oracle.DELOPAR)
        yp = (hM * (yP - yO) / hP + hP * (yO - yM) / hM) / (hM + hP)
        cP_par = yO + 0.5 * hP * yp
        overshoot_OP = not (min(yO, yP) <= cP_par <= max(yO, yP))
        cM_par = yO - 0.5 * hM * yp
        overshoot_MO = not (min(yM, yO) <= cM_par <= max(yM, yO))
        if not overshoot_OP and not overshoot_MO:
            assert cM == pytest.approx(cD, rel=1e-14, abs=1e-14)
        elif overshoot_OP and not overshoot_MO:
            n_clip += 1
            # clipped downwind control point c_P = y_P; derivative at O from the left spline
            dleft = 2 * (yO - cM) / hM
            dright = 2 * (yP - yO) / hP
            assert dleft == pytest.approx(dright, rel=1e-12, abs=1e-12)
    assert n_clip > 50
