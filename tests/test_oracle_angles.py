"""Pins of the oracle's quadratures and spherical tensors T^K_Q(i, Omega) (Eq. 1)."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 10])
def test_gauss_legendre_matches_numpy(n):
    x, w = oracle.gauss_legendre01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, (xr + 1) / 2, rtol=0, atol=2e-15)
    assert np.allclose(w, wr / 2, rtol=0, atol=2e-15)


@pytest.mark.parametrize("n_mu,n_chi", [(3, 8), (5, 16), (4, 10), (2, 3)])
def test_angular_quadrature_moments(n_mu, n_chi):
    atm = synth.plane_parallel_box(2, 2, 4)
    p = oracle.Problem(atm, 0, n_mu, n_chi, 3)
    mu, chi, w = oracle.rays(p)
    assert len(mu) == 2 * n_mu * n_chi
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert (w * mu).sum() == pytest.approx(0.0, abs=1e-15)
    assert (w * mu**2).sum() == pytest.approx(1.0 / 3.0, abs=1e-15)
    ox = np.sqrt(1 - mu**2) * np.cos(chi)
    oy = np.sqrt(1 - mu**2) * np.sin(chi)
    assert abs((w * ox).sum()) < 1e-15 and abs((w * oy).sum()) < 1e-15
    assert (w * ox * ox).sum() == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert (w * oy * oy).sum() == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert abs((w * ox * oy).sum()) < 1e-15


def test_frequency_quadrature():
    x, w = oracle.freqs(11, 4.0)
    assert np.allclose(x, np.linspace(-4, 4, 11))
    assert w.sum() == pytest.approx(8.0)
    assert w[0] == pytest.approx(0.4) and w[5] == pytest.approx(0.8)


def _basis(mu, chi):
    st = math.sqrt(max(0.0, 1 - mu * mu))
    om = np.array([st * math.cos(chi), st * math.sin(chi), mu])
    ea = np.array([mu * math.cos(chi), mu * math.sin(chi), -st])
    eb = np.array([-math.sin(chi), math.cos(chi), 0.0])
    return om, ea, eb


def _spherical2(A):
    """Spherical components A_Q (Q = 0, 1, 2) of a symmetric traceless 3x3 tensor."""
    return np.array([
        math.sqrt(1.5) * A[2, 2],
        -(A[0, 2] + 1j * A[1, 2]),
        0.5 * (A[0, 0] - A[1, 1] + 2j * A[0, 1]),
    ])


def _tkq_cartesian(mu, chi):
    """T^K_Q built from the polarization tensors of the ray frame (e_a, e_b, Omega):
    Stokes I, Q, U <-> e_a e_a + e_b e_b, e_a e_a - e_b e_b, e_a e_b + e_b e_a. The rank-2
    part is -sqrt(3)/2 times the spherical components of the traceless symmetric part
    (the normalization is fixed by the intensity row T^2_0(0) at theta = 0)."""
    om, ea, eb = _basis(mu, chi)
    tens = [np.outer(ea, ea) + np.outer(eb, eb), np.outer(ea, ea) - np.outer(eb, eb),
            np.outer(ea, eb) + np.outer(eb, ea)]
    out = np.zeros((3, 6))
    for i, t in enumerate(tens):
        A = t - np.trace(t) / 3 * np.eye(3)
        s = -math.sqrt(3) / 2 * _spherical2(A)
        out[i] = [np.trace(t) / 2, s[0].real, s[1].real, s[1].imag, s[2].real, s[2].imag]
    return out


def test_tkq_matches_cartesian_construction():
    rng = np.random.default_rng(0)
    for _ in range(200):
        mu = rng.uniform(-1, 1)
        chi = rng.uniform(0, 2 * math.pi)
        assert np.allclose(oracle.tkq(mu, chi), _tkq_cartesian(mu, chi), atol=1e-14)


def test_tkq_vertical_values_and_integrals():
    t = oracle.tkq(1.0, 0.3)
    assert t[0, 0] == 1 and t[0, 1] == pytest.approx(1 / math.sqrt(2))
    assert np.allclose(t[0, 2:], 0) and np.allclose(t[1, :2], 0) and np.allclose(t[2, :2], 0)
    # closed integral over the sphere of the intensity row: delta_K0 delta_Q0
    xg, wg = np.polynomial.legendre.leggauss(20)
    acc = np.zeros((3, 6))
    nchi = 24
    for mu, wm in zip(xg, wg):
        for a in range(nchi):
            acc += wm / 2 / nchi * oracle.tkq(mu, 2 * math.pi * a / nchi)
    assert acc[0, 0] == pytest.approx(1.0)
    assert np.allclose(acc[0, 1:], 0, atol=1e-14)
    # linear-polarization rows along the vertical: only Q = +-2 survives
    t = oracle.tkq(1.0, 0.3)
    e2 = np.exp(2j * 0.3)
    assert complex(t[1, 4], t[1, 5]) == pytest.approx(-math.sqrt(3) / 2 * e2)
    assert complex(t[2, 4], t[2, 5]) == pytest.approx(-1j * math.sqrt(3) / 2 * e2)
    assert np.allclose(t[1:, 1:4], 0)


def _emission(t6, s6):
    """S_i = sum_Q (-1)^Q T^K_Q S^K_{-Q}, the form the oracle uses (Eq. 1 / LL04)."""
    return t6[0] * s6[0] + t6[1] * s6[1] + 2 * (t6[2] * s6[2] + t6[3] * s6[3]) + 2 * (t6[4] * s6[4] + t6[5] * s6[5])


def test_dipole_scattering_of_a_beam():
    """A Jl=0 -> Ju=1 atom (w^(2) = 1) illuminated by an unpolarized beam from Omega'
    re-emits with the Rayleigh phase function 3/4 (1 + cos^2 Theta) and linear
    polarization sin^2 Theta/(1 + cos^2 Theta) perpendicular to the scattering plane."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        mu1, chi1 = rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi)
        mu2, chi2 = rng.uniform(-1, 1), rng.uniform(0, 2 * math.pi)
        J = oracle.tkq(mu1, chi1)[0]            # J^K_Q of a unit beam (Eq. 1)
        t = oracle.tkq(mu2, chi2)
        SI, SQ, SU = (_emission(t[i], J) for i in range(3))
        om1, _, _ = _basis(mu1, chi1)
        om2, ea, eb = _basis(mu2, chi2)
        c = float(om1 @ om2)
        assert SI == pytest.approx(0.75 * (1 + c * c), abs=1e-12)
        p = math.hypot(SQ, SU) / SI
        assert p == pytest.approx((1 - c * c) / (1 + c * c), abs=1e-12)
        if 1 - c * c > 1e-3:
            # electric vector direction psi from e_a: tan 2 psi = U/Q
            psi = 0.5 * math.atan2(SU, SQ)
            evec = math.cos(psi) * ea + math.sin(psi) * eb
            n = np.cross(om1, om2)
            n /= np.linalg.norm(n)
            assert abs(abs(evec @ n) - 1) < 1e-9
