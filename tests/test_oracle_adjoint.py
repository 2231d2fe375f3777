"""Pins of the oracle's adjoint (reverse-mode) sweep of the emergent Stokes vector.

The adjoint is checked against central finite differences of the oracle's own
forward solution (itself pinned by the tests of test_oracle_sweep.py), piece
by piece (step coefficients against mpmath derivatives of the closed forms of
Eqs. 9-13, BESSER control point, 4x4 step) and as a whole on tiny grids.
"""
import numpy as np
import pytest

import oracle
import synth

mpmath = pytest.importorskip("mpmath")


def _closed_forms(t):
    e = mpmath.exp(-t)
    return [e, (1 - e * (1 + t)) / t, (e + t - 1) / t, (2 - e * (t * t + 2 * t + 2)) / t ** 2,
            1 - 2 * (e + t - 1) / t ** 2, 2 * (t - 2 + e * (t + 2)) / t ** 2]


def test_coefficient_derivatives_match_mpmath():
    mpmath.mp.dps = 60
    for t in np.geomspace(1e-7, 300.0, 47):
        ref = [float(mpmath.diff(lambda s, i=i: _closed_forms(s)[i], mpmath.mpf(t))) for i in range(6)]
        got = oracle.coeffs_deriv(t)
        for i in range(6):
            assert abs(got[i] - ref[i]) <= 1e-10 * abs(ref[i]) + 1e-300, (t, i, got[i], ref[i])


def _fd(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


def _branch(yM, yO, yP, hM, hP):
    """Which of steps 2, 6, 7 (clipped) or 4 (parabola) the control point takes."""
    dM, dP = (yO - yM) / hM, (yP - yO) / hP
    if dM * dP <= 0:
        return 2
    yp = (hM * dP + hP * dM) / (hM + hP)
    cM, cP = yO - 0.5 * hM * yp, yO + 0.5 * hP * yp
    if cM < min(yM, yO) or cM > max(yM, yO):
        return 6
    if cP < min(yO, yP) or cP > max(yO, yP):
        return 7
    return 4


@pytest.mark.parametrize("method", [oracle.BESSER, oracle.DELOPAR])
def test_control_point_vjp_matches_finite_differences(method):
    rng = np.random.default_rng(3)
    seen = set()
    for _ in range(400):
        args = list(rng.normal(size=3)) + list(np.exp(rng.normal(size=2)))
        seen.add(_branch(*args))
        g = oracle.control_point_vjp(*args, has_p=True, method=method, gc=1.7)
        for i in range(5):
            def f(v, i=i):
                a = list(args)
                a[i] = v
                return 1.7 * oracle.control_point(*a, has_p=True, method=method)
            h = 1e-6 * max(1.0, abs(args[i]))
            d1, d2 = _fd(f, args[i], h), _fd(f, args[i], h / 4)
            if abs(d1 - d2) > 1e-6 * (1 + abs(d1)):
                continue          # a branch boundary lies within the step
            assert abs(g[i] - d1) <= 1e-6 * (1 + abs(d1)), (args, i, g[i], d1)
    if method == oracle.BESSER:
        assert seen == {2, 4, 6, 7}
    # without a downwind point the control point is the mean of y_M and y_O
    assert np.allclose(oracle.control_point_vjp(0.3, 1.1, 9.0, 0.5, 0.7, has_p=False, gc=2.0), [1, 1, 0, 0, 0])


def _step_inputs(rng, ns, general):
    IM = rng.normal(size=ns)
    etaM = np.zeros(7); etaO = np.zeros(7)
    etaM[0], etaO[0] = np.exp(rng.normal(size=2))
    if ns == 4:
        idx = range(1, 7) if general else [3]
        for q in idx:
            etaM[q] = 0.3 * etaM[0] * rng.normal()
            etaO[q] = 0.3 * etaO[0] * rng.normal()
    epsM = etaM[0] * (1 + 0.3 * rng.normal(size=ns))
    epsO = etaO[0] * (1 + 0.3 * rng.normal(size=ns))
    etaP = float(np.exp(rng.normal()))
    epsP = etaP * (1 + 0.3 * rng.normal(size=ns))
    dsM, dsP = np.exp(rng.normal(size=2))
    return [IM, etaM, epsM, etaO, epsO, etaP, epsP, float(dsM), float(dsP)]


@pytest.mark.parametrize("ns,general,has_p", [(1, False, True), (1, False, False), (4, False, True),
                                              (4, True, True), (4, True, False)])
def test_step_vjp_matches_finite_differences(ns, general, has_p):
    rng = np.random.default_rng(10 + ns + 2 * general + 4 * has_p)
    names = ["IM", "etaM", "epsM", "etaO", "epsO", "etaP", "epsP"]
    checked = 0
    for _ in range(25):
        a = _step_inputs(rng, ns, general)
        gIO = rng.normal(size=ns)
        g = oracle.step_vjp(ns, *a, gIO, has_p=has_p)

        def L(b):
            IO, _ = oracle.step(ns, *b, has_p=has_p)
            return float(gIO @ IO)

        for ai, name in enumerate(names):
            arr = a[ai]
            n = 1 if np.isscalar(arr) or isinstance(arr, float) else len(arr)
            for c in range(n):
                if name in ("etaM", "etaO") and ns == 1 and c > 0:
                    continue
                if name in ("etaM", "etaO") and not general and c not in (0, 3):
                    continue
                if name in ("etaP", "epsP") and not has_p:
                    continue

                def f(v, ai=ai, c=c):
                    b = [x.copy() if isinstance(x, np.ndarray) else x for x in a]
                    if isinstance(b[ai], np.ndarray):
                        b[ai][c] = v
                    else:
                        b[ai] = v
                    return L(b)

                x0 = a[ai][c] if isinstance(a[ai], np.ndarray) else a[ai]
                h = 1e-6 * max(abs(x0), 1e-3)
                d1, d2 = _fd(f, x0, h), _fd(f, x0, h / 4)
                if abs(d1 - d2) > 1e-6 * (1 + abs(d1)):
                    continue
                got = g[name][c] if isinstance(g[name], np.ndarray) else g[name]
                assert abs(got - d1) <= 2e-6 * (1 + abs(d1)), (name, c, got, d1)
                checked += 1
    assert checked > 100


def _params(atm, rho, pol):
    chi = atm["chi"].copy()
    e = chi * rho[..., 0]
    B = np.stack([atm["bx"], atm["by"], atm["bz"]]) if pol else None
    return chi, e, B


def _emergent_of(atm, rho, model, quad, mu, az, chi, e, B):
    """Emergent Stokes at parameters (chi, e, B): the multipoles scale as e/chi with fixed ratios."""
    a = dict(atm)
    a["chi"] = chi
    if B is not None:
        a["bx"], a["by"], a["bz"] = B[0], B[1], B[2]
    r = rho / rho[..., :1] * (e / chi)[..., None]
    p = oracle.Problem(a, model, *quad)
    return oracle.emergent(p, r, mu, az)


@pytest.mark.parametrize("pol", [False, True])
def test_emergent_vjp_matches_finite_differences(pol):
    nx, ny, nz = 4, 3, 6
    if pol:
        atm = synth.random_box(nx, ny, nz, seed=5)
        # a field strong enough that eta_V matters on this tiny grid
        for k in ("bx", "by", "bz"):
            atm[k] = atm[k] * 300.0
    else:
        atm = synth.plane_parallel_box(nx, ny, nz, modulation=0.3)
        atm["vel"] = np.random.default_rng(2).normal(size=atm["chi"].shape)
    model = 1 if pol else 0
    quad = (1, 2, 3)
    rng = np.random.default_rng(7)
    nl = oracle.nl_of(model)
    rho = np.zeros((nz, ny, nx, nl))
    rho[..., 0] = rng.uniform(0.5, 1.5, (nz, ny, nx))
    if nl > 1:
        rho[..., 1:] = 0.05 * rng.normal(size=(nz, ny, nx, nl - 1))
    mu = np.array([1.0, 0.5, 0.7])
    az = np.array([0.0, 0.4, 2.9])
    chi, e, B = _params(atm, rho, pol)
    p = oracle.Problem(atm, model, *quad)
    out = oracle.emergent(p, rho, mu, az)
    gout = rng.normal(size=out.shape)
    g_chi, g_e, g_b = oracle.emergent_vjp(p, rho, mu, az, gout)

    def L(chi_, e_, B_):
        return float(np.sum(gout * _emergent_of(atm, rho, model, quad, mu, az, chi_, e_, B_)))

    checks = [("chi", g_chi), ("e", g_e)] + ([("B", g_b)] if pol else [])
    nchecked = 0
    for name, g in checks:
        scale = np.max(np.abs(g))
        assert scale > 0
        for idx in np.ndindex(g.shape):
            def f(v):
                c2, e2 = chi.copy(), e.copy()
                B2 = B.copy() if B is not None else None
                if name == "chi":
                    c2[idx] = v
                elif name == "e":
                    e2[idx] = v
                else:
                    B2[idx] = v
                return L(c2, e2, B2)
            x0 = {"chi": chi, "e": e, "B": B}[name][idx]
            h = 1e-5 * max(abs(x0), 1e-8 if name != "B" else 1.0)
            d1, d2 = _fd(f, x0, h), _fd(f, x0, h / 4)
            if abs(d1 - d2) > 1e-7 * scale + 1e-5 * abs(d1):
                continue
            assert abs(g[idx] - d1) <= 1e-7 * scale + 1e-5 * abs(d1), (name, idx, g[idx], d1)
            nchecked += 1
    nvox = nx * ny * nz
    assert nchecked >= (0.9 * (5 if pol else 2)) * nvox
    # the bottom boundary plane only enters through the upwind interpolation of plane 1,
    # and every parameter of the grid reaches the top plane along some ray
    assert np.all(np.abs(g_chi[0]) > 0)
