"""Pins of the oracle's reverse mode through Jacobi iterations: the update
(or_see_update_vjp), the J^K_Q / Lambda-bar* of a formal solution
(or_jkq_vjp), the emergent Stokes vector in the unknowns (or_emergent_vjp_rho)
and the checkpointed gradient of an emergent-Stokes loss through iterations
(oracle/diff.py), each against central differences of the pinned forward
routines."""
import numpy as np
import pytest

import oracle
import synth
from oracle import diff


def _atm(nx, ny, nz, pol, seed=1, bscale=1.0):
    if pol:
        a = synth.random_box(nx, ny, nz, seed=seed, tau_top=1e-2, tau_bot=1e2)
        for k in ("bx", "by", "bz"):
            a[k] = a[k] * bscale
    else:
        a = synth.plane_parallel_box(nx, ny, nz, modulation=0.3, tau_top=1e-2, tau_bot=1e2)
        a["vel"] = 0.5 * np.random.default_rng(seed).normal(size=a["chi"].shape)
    a["eps"] = np.full_like(a["eps"], 0.05)
    return a


def _rho(p, atm, seed):
    rng = np.random.default_rng(seed)
    rho = oracle.initial_rho(p, atm) * (1 + 0.2 * rng.uniform(size=p.shape + (1,)))
    if rho.shape[-1] > 1:
        rho[..., 1:] = 0.05 * rho[..., :1] * rng.normal(size=rho[..., 1:].shape)
    return rho


def _check(name, g, f, w, x0, h=1e-3, tol=1e-6, min_frac=0.8):
    """Central differences of L(x) = sum w * f(x) at x0 against g, all
    components, Richardson-extrapolated over the relative steps h and h/2; the
    outputs are differenced before weighting (forming L first would round away
    the change made by a parameter of an optically very thin layer). A component
    whose two differences disagree is skipped -- a BESSER branch changes within
    the step (the map is piecewise smooth); most components must be checked."""
    scale = np.max(np.abs(g)) + 1e-300
    fails = checked = 0
    for i in range(x0.size):
        def cd(step):
            d = np.zeros(x0.size)
            d[i] = step * (abs(x0.flat[i]) if x0.flat[i] != 0 else 1.0)
            return float(np.sum(w * (f(x0 + d.reshape(x0.shape)) - f(x0 - d.reshape(x0.shape))))) / (2 * d[i])
        c1, c2 = cd(h), cd(h / 2)
        if abs(c1 - c2) > 1e-4 * abs(c2) + 0.1 * tol * scale:
            continue
        fd = (4.0 * c2 - c1) / 3.0
        checked += 1
        if abs(fd - g.flat[i]) > tol * scale + 1e-5 * abs(fd):
            fails += 1
    assert fails == 0 and checked >= min_frac * x0.size, (name, fails, checked, x0.size)


def test_see_update_vjp_matches_central_differences():
    atm = _atm(3, 2, 4, True, bscale=20.0)
    quad = (2, 4, 2)
    p = oracle.Problem(atm, 1, *quad)
    rho = _rho(p, atm, 3)
    jkq, ls = oracle.formal_solve(p, rho)
    f = 0.05 * np.asarray(atm["bpl"]) * (1 + 0.1 * np.random.default_rng(4).normal(size=p.shape))
    src = np.zeros(p.shape + (6,)); src[..., 0] = f
    g = np.random.default_rng(5).normal(size=rho.shape)
    gr, gj, gl, gf, gb = oracle.see_update_vjp(p, jkq, ls, rho, g, src)

    def L(rho_=rho, jkq_=jkq, ls_=ls, src_=src, prob=p):
        r, _ = oracle.see_update_src(prob, jkq_, ls_, rho_, src_)
        return r

    _check("rho", gr, lambda x: L(rho_=x), g, rho)
    _check("jkq", gj, lambda x: L(jkq_=x), g, jkq)
    _check("lstar", gl, lambda x: L(ls_=x), g, ls)

    def Lf(x):
        s = src.copy(); s[..., 0] = x
        return L(src_=s)
    _check("f", gf, Lf, g, f)

    def LB(x):
        a = dict(atm); a["bx"], a["by"], a["bz"] = x[0], x[1], x[2]
        return L(prob=oracle.Problem(a, 1, *quad))
    B = np.stack([atm["bx"], atm["by"], atm["bz"]])
    _check("B", gb, LB, g, B)


@pytest.mark.parametrize("pol", [False, True])
def test_jkq_vjp_matches_central_differences(pol):
    atm = _atm(3, 2, 5, pol, bscale=300.0)
    model = 1 if pol else 0
    quad = (1, 2, 2)
    p = oracle.Problem(atm, model, *quad)
    rho = _rho(p, atm, 6)
    jkq, ls = oracle.formal_solve(p, rho)
    rng = np.random.default_rng(7)
    gj, gl = rng.normal(size=jkq.shape), rng.normal(size=ls.shape)
    g_chi, g_rho, g_b = oracle.jkq_vjp(p, rho, gj, gl)

    w = np.concatenate([gj.ravel(), gl.ravel()])

    def L(a=atm, r=rho):
        j, l = oracle.formal_solve(oracle.Problem(a, model, *quad), r)
        return np.concatenate([j.ravel(), l.ravel()])

    def Lchi(x):
        a = dict(atm); a["chi"] = x
        return L(a=a)
    _check("chi", g_chi, Lchi, w, np.asarray(atm["chi"]))
    _check("rho", g_rho, lambda x: L(r=x), w, rho)
    if pol:
        def LB(x):
            a = dict(atm); a["bx"], a["by"], a["bz"] = x[0], x[1], x[2]
            return L(a=a)
        _check("B", g_b, LB, w, np.stack([atm["bx"], atm["by"], atm["bz"]]))


def test_emergent_vjp_rho_matches_differences_and_the_e_parametrization():
    atm = _atm(3, 2, 5, True, bscale=300.0)
    quad = (1, 1, 3)
    p = oracle.Problem(atm, 1, *quad)
    rho = _rho(p, atm, 8)
    mu, az = np.array([1.0, 0.6]), np.array([0.0, 2.0])
    out = oracle.emergent(p, rho, mu, az)
    gout = np.random.default_rng(9).normal(size=out.shape)
    g_chi, g_rho, g_b = oracle.emergent_vjp_rho(p, rho, mu, az, gout)

    def L(a=atm, r=rho):
        return oracle.emergent(oracle.Problem(a, 1, *quad), r, mu, az)

    def Lchi(x):
        a = dict(atm); a["chi"] = x
        return L(a=a)
    _check("chi", g_chi, Lchi, gout, np.asarray(atm["chi"]))
    _check("rho", g_rho, lambda x: L(r=x), gout, rho)
    # the (chi, e) parametrization of the first adjoint follows from this one:
    # rho = (e/chi) r with fixed ratios r -> dL/de = sum_c r_c g_rho_c / chi,
    # dL/dchi|_e = dL/dchi|_rho - sum_c rho_c g_rho_c / chi
    ge_chi, ge_e, ge_b = oracle.emergent_vjp(p, rho, mu, az, gout)
    chi = np.asarray(atm["chi"])
    assert np.allclose(ge_e, np.sum(rho / rho[..., :1] * g_rho, -1) / chi, rtol=1e-10, atol=1e-14 * np.abs(ge_e).max())
    assert np.allclose(ge_chi, g_chi - np.sum(rho * g_rho, -1) / chi, rtol=1e-10, atol=1e-12 * np.abs(ge_chi).max())
    assert np.allclose(ge_b, g_b, rtol=1e-12, atol=0)


@pytest.mark.parametrize("pol", [False, True])
def test_gradient_through_iterations_matches_central_differences(pol):
    atm = _atm(4, 2, 6, pol, seed=3, bscale=50.0)
    # a varying Planck function: with S = B = 1 everywhere the first iterates are
    # nearly uniform and the control points sit on BESSER's step-2 kink
    atm["bpl"] = np.exp(0.3 * np.random.default_rng(11).normal(size=atm["chi"].shape))
    model = 1 if pol else 0
    quad = (2, 4, 3)
    mu, az = np.array([1.0, 0.5]), np.array([0.0, 1.0])
    f0 = np.asarray(atm["eps"]) * np.asarray(atm["bpl"])
    tatm = _atm(4, 2, 6, pol, seed=4, bscale=50.0)
    tatm["bpl"] = atm["bpl"]
    _, target = diff.forward(tatm, model, quad, np.asarray(tatm["eps"]) * np.asarray(tatm["bpl"]), 3, mu, az)
    L, g_chi, g_f, g_b, _ = diff.loss_and_grad(atm, model, quad, f0, 3, 2, mu, az, target)

    def loss(a, f):
        _, o = diff.forward(a, model, quad, f, 3, mu, az)
        return o

    def check(name, make, x0, g, h=1e-5, signed=False):
        """Richardson-extrapolated central differences of the quadratic loss, formed
        exactly from the outputs (sum (o+ - o-)(o+ + o- - 2 t)). A sample is rejected
        only where a BESSER control point changes branch inside the interval (the
        piecewise-smooth control point of Sec. 3.2, where a difference is not a
        derivative): the oracle's branch signature at x0 +- h and x0 +- h/2 must equal
        the one at x0. The rejected components are reported; at least 80 % are kept."""
        _, sig0 = oracle.branch_signature(make, x0)
        scale = np.max(np.abs(g))
        # steps relative to each component; for a signed parameter (the field)
        # at least relative to its RMS, since a step relative to a near-zero
        # component is lost in the outputs' rounding
        xs = np.sqrt(np.mean(x0 ** 2)) if signed else 0.0
        fails, rejected, worst = [], [], 0.0
        for i in range(x0.size):
            sigs = []

            def cd(step):
                d = step * max(abs(x0.flat[i]), xs)
                xp, xm = x0.copy(), x0.copy()
                xp.flat[i] += d; xm.flat[i] -= d
                op, sp = oracle.branch_signature(make, xp)
                om, sm = oracle.branch_signature(make, xm)
                sigs.extend([sp, sm])
                return np.sum((op - om) * (op + om - 2 * target)) / (2 * d)
            c1, c2 = cd(h), cd(h / 2)
            if any(s != sig0 for s in sigs):
                rejected.append(i)
                continue
            err = abs((4 * c2 - c1) / 3 - g.flat[i]) / (scale + abs(c2))
            worst = max(worst, err)
            if err > 1e-6:
                fails.append((i, err))
        kept = x0.size - len(rejected)
        print(f"{name}: kept {kept}/{x0.size}, rejected (branch change) {rejected}, worst {worst:.2e}")
        assert not fails and kept >= 0.8 * x0.size, (name, fails, rejected, x0.size)

    def with_chi(x):
        a = dict(atm); a["chi"] = x
        return loss(a, f0)
    check("chi", with_chi, np.asarray(atm["chi"]), g_chi)
    check("f", lambda x: loss(atm, x), f0, g_f)
    if pol:
        def with_b(x):
            a = dict(atm); a["bx"], a["by"], a["bz"] = x[0], x[1], x[2]
            return loss(a, f0)
        check("B", with_b, np.stack([atm["bx"], atm["by"], atm["bz"]]), g_b, signed=True)
    # checkpoint spacing does not change the result
    L2, c2, f2, b2, _ = diff.loss_and_grad(atm, model, quad, f0, 3, 1, mu, az, target)
    assert L2 == L and np.array_equal(c2, g_chi) and np.array_equal(f2, g_f) and np.array_equal(b2, g_b)
