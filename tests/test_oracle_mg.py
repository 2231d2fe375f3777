"""Pins of the oracle's multigrid pieces: transfer operators (Sec. 5.2), the
statistical-equilibrium operator A and its Jacobi update with a source term,
and the FAS V-cycle (Sec. 5.1), against definitions, brute force and the
Jacobi fixed point."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mg


def _atm(nx, ny, nz, pol, seed=1):
    if pol:
        return synth.random_box(nx, ny, nz, seed=seed, tau_top=1e-2, tau_bot=1e2)
    a = synth.plane_parallel_box(nx, ny, nz, modulation=0.3, tau_top=1e-2, tau_bot=1e2)
    a["vel"] = 0.5 * np.random.default_rng(seed).normal(size=a["chi"].shape)
    return a


@pytest.mark.parametrize("nz", [9, 8])
def test_prolongation_injects_and_interpolates_linearly(nz):
    atm = _atm(6, 4, nz, False)
    lev = mg.Level(atm, 0, (1, 2, 2))
    nc = mg.coarse_nz(nz)
    zc = np.asarray(atm["z"])[0:2 * nc:2]
    rng = np.random.default_rng(0)
    c = rng.normal(size=(nc, 2, 3, 2))
    f = mg.prolong(lev, c)
    assert np.array_equal(f[0::2, 0::2, 0::2][:nc], c)                 # coarse nodes: injection
    # midpoints in x and y: the mean of the two neighbours (periodic)
    assert np.allclose(f[0:2 * nc:2, 0::2, 1::2], 0.5 * (c + np.roll(c, -1, axis=2)))
    assert np.allclose(f[0:2 * nc:2, 1::2, 0::2], 0.5 * (c + np.roll(c, -1, axis=1)))
    # a field linear in z (constant horizontally) is reproduced exactly, also
    # by the extrapolated top plane of an even number of planes
    lin = np.broadcast_to((2.0 + 3.0 * zc)[:, None, None, None], (nc, 2, 3, 1))
    ref = np.broadcast_to((2.0 + 3.0 * np.asarray(atm["z"]))[:, None, None, None], (nz, 4, 6, 1))
    assert np.allclose(mg.prolong(lev, lin), ref, rtol=1e-13)


@pytest.mark.parametrize("nz", [9, 8])
def test_restriction_is_the_normalized_transpose_of_prolongation(nz):
    atm = _atm(4, 6, nz, False)
    lev = mg.Level(atm, 0, (1, 2, 2))
    nc = mg.coarse_nz(nz)
    cs, fs = (nc, 3, 2, 1), (nz, 6, 4, 1)
    # dense P by brute force: prolong every coarse unit vector
    Pd = np.zeros((int(np.prod(fs)), int(np.prod(cs))))
    for j in range(Pd.shape[1]):
        e = np.zeros(Pd.shape[1]); e[j] = 1.0
        Pd[:, j] = mg.prolong(lev, e.reshape(cs)).ravel()
    u = np.random.default_rng(1).normal(size=fs)
    Ru = mg.restrict(lev, u).ravel()
    assert np.allclose(Ru, (Pd.T @ u.ravel()) / Pd.sum(0), rtol=1e-13)
    assert np.allclose(mg.restrict(lev, np.full(fs, 2.5)), 2.5, rtol=1e-14)
    # horizontally: full weighting 1/4, 1/2, 1/4 per axis (periodic)
    Py = mg.prolong_1d_periodic(6)
    assert np.allclose((Py.T / Py.sum(0)[:, None])[1], [0, 0.25, 0.5, 0.25, 0, 0])
    assert np.allclose((Py.T / Py.sum(0)[:, None])[0], [0.5, 0.25, 0, 0, 0, 0.25])


@pytest.mark.parametrize("pol", [False, True])
def test_see_apply_and_source_term_update(pol):
    atm = _atm(4, 4, 7, pol)
    model = 1 if pol else 0
    quad = (2, 4, 3)
    p = oracle.Problem(atm, model, *quad)
    rho = oracle.initial_rho(p, atm) * (1.0 + 0.1 * np.random.default_rng(2).normal(size=(7, 4, 4, 1)))
    if pol:
        rho[..., 1:] = 0.02 * np.random.default_rng(3).normal(size=rho[..., 1:].shape)
    jkq, ls = oracle.formal_solve(p, rho)
    # the source-term update with src = eps B delta_K0 is the two-level update
    lev = mg.Level(atm, model, quad)
    f = mg.f_fine(lev)
    r1, m1 = oracle.see_update(p, jkq, ls, rho)
    r2, m2 = oracle.see_update_src(p, jkq, ls, rho, f)
    assert np.array_equal(r1, r2) and m1 == m2
    # A written out: S - (1-eps) J for K = 0; for K = 2 the Hanle matrix applied to S^2,
    # checked through the Hanle solve: solving M x = A(S)^2 + (1-eps) J^2 returns S^2
    A = oracle.see_apply(p, jkq, rho)
    e = np.asarray(atm["eps"])
    assert np.allclose(A[..., 0], rho[..., 0] - (1 - e) * jkq[..., 0], rtol=1e-14)
    if pol:
        B = np.stack([atm["bx"], atm["by"], atm["bz"]], -1)
        for idx in [(0, 0, 0), (3, 2, 1), (6, 3, 3)]:
            gam = -(1 - e[idx]) * np.linalg.norm(B[idx]) / atm["bcrit"]      # the -i of the magnetic term
            x = oracle.hanle_solve(gam, B[idx], A[idx] + (1 - e[idx]) * jkq[idx])
            assert np.allclose(x[1:], rho[idx][1:], rtol=1e-12, atol=1e-15)
    # Jacobi with a general source converges to a solution of A(S) = src
    src = f + 0.05 * np.abs(f).max() * np.random.default_rng(4).uniform(size=f.shape)
    r, mc = mg.jacobi(lev, rho, src, 200)
    assert mc < 1e-12
    assert np.max(np.abs(mg.apply_A(lev, r) - src)) < 1e-10 * np.max(np.abs(src))


def _residual(level, rho):
    f = mg.f_fine(level)
    return np.max(np.abs(f - mg.apply_A(level, rho))) / np.max(np.abs(f))


@pytest.mark.parametrize("pol,nz", [(False, 33), (True, 32)])
def test_vcycles_solve_the_fine_grid_equations(pol, nz):
    # 8 planes per decade of optical depth on the finest grid, 2 on the coarsest
    # (the method needs the coarse grids to resolve the transfer problem, Sec. 5.3)
    atm = _atm(8, 8, nz, pol, seed=5)
    atm["eps"] = np.full_like(atm["eps"], 1e-2)
    model = 1 if pol else 0
    quad = (2, 4, 3)
    levels = mg.hierarchy(atm, model, quad, 3)
    nc = mg.coarse_nz(nz)
    assert [l.shape for l in levels] == [(nz, 8, 8), (nc, 4, 4), (mg.coarse_nz(nc), 2, 2)]
    fine = levels[0]
    rho0 = oracle.initial_rho(fine.prob, atm)
    # Jacobi with the same number of fine-grid formal solutions as 4 V-cycles
    # (2 + 4 smoothing sweeps and one residual per cycle)
    rj, _ = mg.jacobi(fine, rho0, None, 4 * 7)
    rho = rho0.copy()
    res = [_residual(fine, rho)]
    for _ in range(4):
        rho = mg.vcycle(levels, rho)
        res.append(_residual(fine, rho))
    assert res[-1] < 3e-2 * _residual(fine, rj)
    assert res[4] < 5e-3 * res[1]          # ~0.15 per cycle (Jacobi of equal cost: ~0.35)
    # the fixed point of the V-cycle solves the fine-grid equations A(rho) = f
    for _ in range(10):
        rho = mg.vcycle(levels, rho)
    assert _residual(fine, rho) < 1e-8      # K=0 shrinks ~5x per cycle, K=2 ~2.5x


@pytest.mark.parametrize("nz", [17, 16])
def test_cubic_prolongation_reproduces_cubics_in_height(nz):
    """Tri-cubic-centered prolongation (Sec. 5.2): a field cubic in z (constant
    horizontally) is reproduced at every fine plane, the extrapolated top one included."""
    atm = _atm(8, 8, nz, False)
    lev = mg.Level(atm, 0, (1, 2, 2))
    nc = mg.coarse_nz(nz)
    z = np.asarray(atm["z"])
    u = (z - z.mean()) / (z.max() - z.min())
    poly = lambda s: 0.3 - 1.2 * s + 0.7 * s ** 2 + 2.1 * s ** 3
    c = np.broadcast_to(poly(u[0:2 * nc:2])[:, None, None, None], (nc, 4, 4, 1))
    ref = np.broadcast_to(poly(u)[:, None, None, None], (nz, 8, 8, 1))
    assert np.allclose(mg.prolong(lev, c, 3), ref, rtol=0, atol=1e-12)
    # the tri-linear operator does not (the field is not linear)
    assert np.max(np.abs(mg.prolong(lev, c, 1) - ref)) > 1e-3


def test_cubic_prolongation_horizontal_stencil():
    nf = 16
    P = mg.prolong_1d_periodic_cubic(nf)
    assert np.allclose(P.sum(1), 1.0)                          # constants are kept
    assert np.array_equal(P[0::2], np.eye(nf // 2))           # injection at coarse nodes
    xc = np.arange(nf // 2, dtype=np.float64)
    xf = np.arange(nf) / 2.0
    cub = lambda x: 1.0 + 0.5 * x - 0.25 * x ** 2 + 0.05 * x ** 3
    got = P @ cub(xc)
    # exact where the four coarse nodes do not wrap around the period
    inner = [i for i in range(1, nf, 2) if 1 <= (i - 1) // 2 <= nf // 2 - 3]
    assert np.allclose(got[inner], cub(xf[inner]), rtol=0, atol=1e-12)
    # fourth order on a smooth periodic field: the error falls 16x per refinement
    err = []
    for n in (16, 32, 64):
        xc = np.arange(n // 2) * 2 * np.pi / (n // 2)
        xf = np.arange(n) * 2 * np.pi / n
        err.append(np.max(np.abs(mg.prolong_1d_periodic_cubic(n) @ np.sin(xc) - np.sin(xf))))
    assert err[0] / err[1] == pytest.approx(16.0, rel=0.1)
    assert err[1] / err[2] == pytest.approx(16.0, rel=0.05)


def test_nested_multigrid_and_cubic_vcycles():
    """The nested method (Sec. 5.1) starts each level from the prolonged coarser
    solution: one cycle per level leaves a smaller fine residual than one V-cycle from
    S = B, and the cycles with either prolongation converge to A(rho) = f."""
    atm = _atm(16, 16, 33, False, seed=5)
    atm["eps"] = np.full_like(atm["eps"], 1e-2)
    quad = (2, 4, 3)
    levels = mg.hierarchy(atm, 0, quad, 3)
    fine, coarsest = levels[0], levels[-1]
    rho0 = oracle.initial_rho(fine.prob, atm)
    r_v1 = _residual(fine, mg.vcycle(levels, rho0.copy(), order=3))
    rho = mg.nested(levels, oracle.initial_rho(coarsest.prob, coarsest.atm), ncycles=1, order=3)
    r_n1 = _residual(fine, rho)
    assert r_n1 < r_v1, (r_n1, r_v1)
    for order in (3, 1):
        r = rho.copy()
        for _ in range(12):
            r = mg.vcycle(levels, r, order=order)
        assert _residual(fine, r) < 1e-8, order
