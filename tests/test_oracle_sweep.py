"""Pins of the oracle's 3D short-characteristics formal solution and Jacobi
iteration against closed forms, symmetries, the 1D solver, and brute force."""
import math

import numpy as np
import pytest

import oracle
import synth


def _uniform_atm(nx, ny, nz, chi=1.0, dz=1.0, lx=None, ly=None, eps=0.1, bpl=1.0, pol=False, bfield=(0, 0, 0)):
    shape = (nz, ny, nx)
    a = dict(nx=nx, ny=ny, nz=nz, lx=lx or nx * 1.0, ly=ly or ny * 1.0, z=np.arange(nz) * dz,
             chi=np.full(shape, chi), eps=np.full(shape, eps), bpl=np.full(shape, bpl),
             vel=np.zeros(shape), zeta=3.5e-4, gbar=1.0, bcrit=25.0)
    if pol:
        a["bx"], a["by"], a["bz"] = (np.full(shape, float(b)) for b in bfield)
    return a


def _tau_along_ray(atm, x, mu, k_order):
    """Trapezoid optical depth between successive planes along a ray (horizontally homogeneous box)."""
    z = atm["z"][k_order]
    eta = atm["chi"][k_order, 0, 0] * math.exp(-x * x)
    dtau = 0.5 * (eta[1:] + eta[:-1]) * np.abs(np.diff(z)) / abs(mu)
    return np.concatenate([[0.0], np.cumsum(dtau)])


def test_constant_source_is_exact_and_thick_medium_gives_I_equal_S():
    """Constant S: I = S (1 - e^-tau) + I_bc e^-tau exactly; deep inside a thick medium I = S."""
    atm = _uniform_atm(3, 3, 30, chi=2.0, dz=1.0, bpl=0.7)
    p = oracle.Problem(atm, 0, 3, 8, 5)
    rho = np.full(p.shape + (1,), 0.7)
    mu, chi, w = oracle.rays(p)
    xf, _ = oracle.freqs(5, 4.0)
    for m in [0, 10, 30, 47]:
        for j in [0, 2]:
            I, ls = oracle.sweep_ray(p, rho, m, j)
            order = np.arange(30) if mu[m] > 0 else np.arange(29, -1, -1)
            tau = _tau_along_ray(atm, xf[j], mu[m], order)
            ibc = 0.7 if mu[m] > 0 else 0.0
            exact = 0.7 * (1 - np.exp(-tau)) + ibc * np.exp(-tau)
            got = I[order, 1, 2, 0]
            assert np.allclose(got, exact, rtol=1e-13, atol=1e-15)
    # opaque at every frequency kept (|x| <= 1, tau >= 70 per level): deep inside, J = S
    thick = _uniform_atm(3, 3, 30, chi=200.0, dz=1.0, bpl=0.7)
    pt = oracle.Problem(thick, 0, 3, 8, 5, x_max=1.0)
    jkq, ls = oracle.formal_solve(pt, rho)
    assert np.allclose(jkq[:20, ..., 0], 0.7, rtol=1e-12)


def test_linear_source_is_exact_for_every_ray():
    """S linear in the vertical optical depth with the matching lower boundary:
    I = a + b tau_v + b |mu|/phi exactly (Eddington-Barbier without error)."""
    nz = 24
    atm = _uniform_atm(2, 3, nz, chi=1.5, dz=0.7)
    z = atm["z"]
    tau_v = 1.5 * (z[-1] - z)          # vertical line-centre optical depth from the top
    a0, b0 = 0.3, 0.8
    p = oracle.Problem(atm, 0, 3, 6, 5)
    mu, _, _ = oracle.rays(p)
    xf, _ = oracle.freqs(5, 4.0)
    rho = np.broadcast_to((a0 + b0 * tau_v)[:, None, None, None], p.shape + (1,)).copy()
    for m in range(0, 18, 4):          # upward rays
        for j in [1, 2]:
            ph = math.exp(-xf[j] ** 2)
            exact = a0 + b0 * tau_v + b0 * abs(mu[m]) / ph
            atm2 = dict(atm)
            atm2["bpl"] = np.broadcast_to(exact[:, None, None], p.shape).copy()
            p2 = oracle.Problem(atm2, 0, 3, 6, 5)
            I, _ = oracle.sweep_ray(p2, rho, m, j)
            assert np.allclose(I[:, 0, 1, 0], exact, rtol=1e-12)


def test_horizontally_homogeneous_box_equals_1d_solution():
    rng = np.random.default_rng(0)
    nz = 20
    atm = _uniform_atm(3, 2, nz, dz=1.0)
    atm["z"] = np.cumsum(rng.uniform(0.3, 1.5, nz))
    chi_z = np.exp(rng.normal(size=nz))
    atm["chi"] = np.broadcast_to(chi_z[:, None, None], (nz, 2, 3)).copy()
    S_z = 1 + 0.5 * np.sin(np.arange(nz)) + rng.uniform(0, 0.3, nz)
    atm["bpl"] = np.full((nz, 2, 3), 1.3)
    p = oracle.Problem(atm, 0, 3, 4, 3)
    rho = np.broadcast_to(S_z[:, None, None, None], p.shape + (1,)).copy()
    mu, _, _ = oracle.rays(p)
    xf, _ = oracle.freqs(3, 4.0)
    for m in range(p.nray):
        for j in range(3):
            I, _ = oracle.sweep_ray(p, rho, m, j)
            order = np.arange(nz) if mu[m] > 0 else np.arange(nz - 1, -1, -1)
            tau = _tau_along_ray(atm, xf[j], mu[m], order)
            ref = oracle.solve_1d(tau, S_z[order], 1.3 if mu[m] > 0 else 0.0)
            for jj in range(2):
                for ii in range(3):
                    assert np.allclose(I[order, jj, ii, 0], ref, rtol=1e-13, atol=1e-16)


def _rand_atm(nx, ny, nz, seed, pol=False):
    a = synth.random_box(nx, ny, nz, seed=seed) if pol else synth.plane_parallel_box(nx, ny, nz)
    if not pol:
        rng = np.random.default_rng(seed)
        a["chi"] = a["chi"] * np.exp(0.3 * rng.normal(size=a["chi"].shape))
        a["vel"] = rng.normal(size=a["chi"].shape)
    return a


def _rand_rho(p, seed):
    rng = np.random.default_rng(seed)
    nl = oracle.nl_of(p.model)
    rho = np.zeros(p.shape + (nl,))
    rho[..., 0] = rng.uniform(0.5, 1.5, p.shape)
    if nl > 1:
        rho[..., 1:] = 0.05 * rng.normal(size=p.shape + (nl - 1,))
    return rho


@pytest.mark.parametrize("pol", [False, True])
def test_translation_invariance(pol):
    """Shifting the periodic atmosphere by whole cells shifts the solution."""
    atm = _rand_atm(5, 4, 6, seed=1, pol=pol)
    p = oracle.Problem(atm, 1 if pol else 0, 2, 4, 5)
    rho = _rand_rho(p, 2)
    jkq, ls = oracle.formal_solve(p, rho)
    sx, sy = 2, 3
    atm2 = {k: (np.roll(v, (sy, sx), axis=(1, 2)) if isinstance(v, np.ndarray) and v.ndim == 3 else v)
            for k, v in atm.items()}
    p2 = oracle.Problem(atm2, p.model, 2, 4, 5)
    jkq2, ls2 = oracle.formal_solve(p2, np.roll(rho, (sy, sx), axis=(1, 2)))
    assert np.allclose(np.roll(jkq, (sy, sx), axis=(1, 2)), jkq2, rtol=1e-12, atol=1e-15)
    assert np.allclose(np.roll(ls, (sy, sx), axis=(1, 2)), ls2, rtol=1e-12, atol=1e-15)


def test_mirror_symmetry_unpolarized():
    """Mirroring x maps azimuth chi to pi - chi: the mirrored problem has the mirrored J."""
    atm = _rand_atm(6, 5, 6, seed=3)
    p = oracle.Problem(atm, 0, 2, 8, 3)
    rho = _rand_rho(p, 4)
    jkq, ls = oracle.formal_solve(p, rho)
    mir = lambda v: np.roll(v[:, :, ::-1], 1, axis=2)     # x_i -> x_{-i}
    atm2 = {k: (mir(v) if isinstance(v, np.ndarray) and v.ndim == 3 else v) for k, v in atm.items()}
    p2 = oracle.Problem(atm2, 0, 2, 8, 3)
    jkq2, ls2 = oracle.formal_solve(p2, mir(rho))
    assert np.allclose(mir(jkq), jkq2, rtol=1e-12)
    assert np.allclose(mir(ls), ls2, rtol=1e-12)


def test_characteristic_through_nodes_equals_1d():
    """If the horizontal displacement between planes is an integer number of cells,
    M and P fall on grid nodes and the 3D solution along the characteristic is the 1D
    solution on that sequence of nodes (periodic wrap included)."""
    nx, ny, nz = 7, 5, 12
    rng = np.random.default_rng(11)
    atm = _uniform_atm(nx, ny, nz, dz=1.0, lx=7.0, ly=5.0)
    atm["chi"] = np.exp(rng.normal(size=(nz, ny, nx)))
    S = rng.uniform(0.5, 2, size=(nz, ny, nx))
    p = oracle.Problem(atm, 0, 3, 8, 3)
    mu, chi, _ = oracle.rays(p)
    m = 1                                   # upward ray, chi = 3 pi / 8
    ox = math.sqrt(1 - mu[m] ** 2) * math.cos(chi[m])
    oy = math.sqrt(1 - mu[m] ** 2) * math.sin(chi[m])
    # choose vertical spacing and cell sizes so that the x shift is 1 cell and the y shift 2 cells
    dz = 1.0
    atm["lx"] = nx * dz * ox / mu[m] / 1.0
    atm["ly"] = ny * dz * oy / mu[m] / 2.0
    p = oracle.Problem(atm, 0, 3, 8, 3)
    rho = S[..., None]
    xf, _ = oracle.freqs(3, 4.0)
    I, _ = oracle.sweep_ray(p, rho, m, 1)
    for i0 in range(nx):
        for j0 in range(ny):
            idx = [((i0 + k) % nx, (j0 + 2 * k) % ny, k) for k in range(nz)]
            eta = np.array([atm["chi"][k, j, i] for i, j, k in idx]) * math.exp(-xf[1] ** 2)
            tau = np.concatenate([[0], np.cumsum(0.5 * (eta[1:] + eta[:-1]) * dz / mu[m])])
            s = np.array([S[k, j, i] for i, j, k in idx])
            ref = oracle.solve_1d(tau, s, atm["bpl"][0, j0, i0])
            got = np.array([I[k, j, i, 0] for i, j, k in idx])
            assert np.allclose(got, ref, rtol=1e-12)


def test_polarized_thick_homogeneous_isotropy():
    """B = 0 and constant S^0_0 in a thick medium: deep voxels see I = S for all rays,
    so J^0_0 = S, J^2_Q = 0 (isotropy invariants of the quadrature)."""
    atm = _uniform_atm(2, 2, 40, chi=300.0, dz=1.0, bpl=0.9, pol=True, bfield=(0, 0, 0))
    p = oracle.Problem(atm, 1, 5, 16, 7, x_max=1.0)
    rho = np.zeros(p.shape + (6,))
    rho[..., 0] = 0.9
    jkq, ls = oracle.formal_solve(p, rho)
    assert np.allclose(jkq[:8, ..., 0], 0.9, rtol=1e-12)
    assert np.allclose(jkq[:8, ..., 1:], 0.0, atol=1e-13)


def test_unno_rachkovsky_constant_matrix_linear_source():
    """Constant propagation matrix K (all seven elements) and a source vector linear in
    optical depth: the exact solution is linear, I = K~^-1 S0 - K~^-2 S1 + K~^-1 S1 s
    (s = optical path along the ray), and the BESSER-DELO step reproduces it exactly."""
    rng = np.random.default_rng(2)
    for trial in range(20):
        pol = rng.normal(size=3)
        pol *= rng.uniform(0.1, 0.9) / np.linalg.norm(pol)
        eta = np.array([1.0, *pol, *(rng.normal(size=3) * 0.7)])
        eI, eQ, eU, eV, rQ, rU, rV = eta
        Kt = np.array([[eI, eQ, eU, eV], [eQ, eI, rV, -rU], [eU, -rV, eI, rQ], [eV, rU, -rQ, eI]])
        S0 = rng.normal(size=4)
        S0[0] += 3
        S1 = rng.normal(size=4) * 0.3
        Ki = np.linalg.inv(Kt)
        exact = lambda s: Ki @ S0 - Ki @ Ki @ S1 + (Ki @ S1) * s
        h = rng.uniform(0.05, 2.0)
        n = 15
        s = np.arange(n) * h
        I = exact(s[0])
        for i in range(1, n):
            has_p = i + 1 < n
            Sp = S0 + S1 * s[i + 1] if has_p else np.zeros(4)
            I, _ = oracle.step(4, I, eta, S0 + S1 * s[i - 1], eta, S0 + S1 * s[i], 1.0, Sp, h, h, has_p)
            assert np.allclose(I, exact(s[i]), rtol=1e-11, atol=1e-12), (trial, i)


def test_sqrt_eps_law():
    """Isothermal semi-infinite two-level atom: S(0) = sqrt(eps) B (plane-parallel box)."""
    atm = synth.plane_parallel_box(1, 1, 32, modulation=0.0)
    p = oracle.Problem(atm, 0, 3, 8, 11)
    rho, hist = oracle.jacobi(p, atm, tol=1e-8, max_iter=3000)
    assert hist[-1] < 1e-8
    s_top = rho[-1, 0, 0, 0]
    err32 = abs(s_top / math.sqrt(1e-2) - 1)
    assert err32 < 2e-2, s_top
    # the residual is spatial discretization: it shrinks as the levels are refined
    atm = synth.plane_parallel_box(1, 1, 64, modulation=0.0)
    p = oracle.Problem(atm, 0, 3, 8, 11)
    rho, hist = oracle.jacobi(p, atm, tol=1e-8, max_iter=3000)
    err64 = abs(rho[-1, 0, 0, 0] / math.sqrt(1e-2) - 1)
    assert err64 < err32 / 4


def test_unmodulated_box_columns_identical():
    atm = synth.plane_parallel_box(4, 4, 16, modulation=0.0)
    p = oracle.Problem(atm, 0, 3, 8, 5)
    rho = oracle.initial_rho(p, atm)
    for _ in range(3):
        jkq, ls = oracle.formal_solve(p, rho)
        rho, _ = oracle.see_update(p, jkq, ls, rho)
    ref = rho[:, :1, :1, :]
    assert np.allclose(rho, ref, rtol=1e-13)


def test_brute_force_newton_matches_jacobi_fixed_point():
    """Solve S - (1-eps) J[S] - eps B = 0 on a 4x4x8 grid by Newton's method with a
    finite-difference Jacobian; the Jacobi (ALI) iteration must reach the same S."""
    atm = synth.plane_parallel_box(4, 4, 8, modulation=0.2, eps=0.1)
    p = oracle.Problem(atm, 0, 2, 4, 5)
    e = atm["eps"].ravel()
    B = atm["bpl"].ravel()

    def F(S):
        jkq, _ = oracle.formal_solve(p, S.reshape(p.shape + (1,)))
        return S - (1 - e) * jkq.ravel() - e * B

    S = B.copy()
    n = S.size
    for it in range(8):
        f = F(S)
        if np.max(np.abs(f)) < 1e-13:
            break
        Jm = np.empty((n, n))
        for i in range(n):
            h = 1e-7 * max(1.0, abs(S[i]))
            Sp = S.copy(); Sp[i] += h
            Jm[:, i] = (F(Sp) - f) / h
        S = S - np.linalg.solve(Jm, f)
    assert np.max(np.abs(F(S))) < 1e-12
    rho, hist = oracle.jacobi(p, atm, tol=1e-13, max_iter=2000)
    assert np.allclose(rho.ravel(), S, rtol=1e-10)


def test_emergent_matches_1d_for_homogeneous_layers():
    rng = np.random.default_rng(5)
    nz = 16
    atm = _uniform_atm(3, 3, nz, dz=1.0, pol=True, bfield=(0, 0, 0))
    chi_z = np.exp(rng.normal(size=nz))
    atm["chi"] = np.broadcast_to(chi_z[:, None, None], (nz, 3, 3)).copy()
    p = oracle.Problem(atm, 1, 2, 4, 5)
    rho = np.zeros(p.shape + (6,))
    S_z = rng.uniform(0.5, 1.5, nz)
    rho[..., 0] = S_z[:, None, None]
    xf, _ = oracle.freqs(5, 4.0)
    mus, chis = np.array([1.0, 0.5, 0.3]), np.array([0.0, 1.0, 4.0])
    out = oracle.emergent(p, rho, mus, chis)
    for d in range(3):
        for j in range(5):
            tau = _tau_along_ray(atm, xf[j], mus[d], np.arange(nz))
            ref = oracle.solve_1d(tau, S_z, atm["bpl"][0, 0, 0])
            assert np.allclose(out[d, j, ..., 0], ref[-1], rtol=1e-13)
            assert np.allclose(out[d, j, ..., 1:], 0.0, atol=1e-15)


def test_jacobi_convergence_rate_is_that_of_delopar():
    """Fig. 4: the Jacobi iteration converges at the same rate with BESSER as with
    DELOPAR: the asymptotic reduction factor of the maximum change per iteration,
    which the approximate operator Lambda* of each step (Eq. 14 for BESSER) sets,
    agrees within 2 %."""
    atm = synth.plane_parallel_box(2, 2, 40, modulation=0.0, eps=1e-3)
    rates = {}
    for meth in (oracle.BESSER, oracle.DELOPAR):
        p = oracle.Problem(atm, 0, 3, 4, 5, method=meth)
        rho = np.zeros((40, 2, 2, 1))
        rho[..., 0] = atm["bpl"]
        ch = []
        for _ in range(40):
            J, L = oracle.formal_solve(p, rho)
            rho, c = oracle.see_update(p, J, L, rho)
            ch.append(c)
        ch = np.array(ch)
        rates[meth] = np.mean(ch[-10:] / ch[-11:-1])
    assert 0.5 < rates[oracle.BESSER] < 0.95
    assert rates[oracle.BESSER] == pytest.approx(rates[oracle.DELOPAR], rel=0.02)
