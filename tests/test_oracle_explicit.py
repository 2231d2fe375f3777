"""Pin of the oracle's sweep with a general propagation matrix (all seven
elements of Eqs. 7-8, an explicit medium): in a thick horizontally homogeneous
slab of constant opacity with a constant K'/eta_I and a source vector linear in
height, the emergent Stokes vector of every direction and frequency is the
Unno-Rachkovsky solution I = (1 + K')^-1 S(z_top) - (1 + K')^-2 (dS/dz) mu / eta_I
(the bottom boundary is forgotten through the slab's optical thickness)."""
import numpy as np

import oracle


def _kprime(k):
    q, u, v, rq, ru, rv = k
    return np.array([[0, q, u, v], [q, 0, rv, -ru], [u, -rv, 0, rq], [v, ru, -rq, 0]], dtype=np.float64)


def explicit_slab(k6, A, Bp, nx=2, ny=2, nz=40, chi=10.0, dz=1.0):
    z = dz * np.arange(nz, dtype=np.float64)
    shape = (nz, ny, nx)
    atm = dict(nx=nx, ny=ny, nz=nz, lx=10.0, ly=10.0, z=z, chi=np.full(shape, chi), eps=np.full(shape, 1e-2),
               bpl=np.full(shape, 1.0), vel=np.zeros(shape), bx=np.zeros(shape), by=np.zeros(shape),
               bz=np.zeros(shape), zeta=0.0, gbar=1.0, bcrit=25.0)
    atm["kexpl"] = np.broadcast_to(np.asarray(k6, dtype=np.float64)[:, None, None, None], (6,) + shape).copy()
    S = np.asarray(A)[:, None] + np.asarray(Bp)[:, None] * z[None, :]
    atm["sexpl"] = np.broadcast_to(S[:, :, None, None], (4,) + shape).copy()
    return atm


def test_explicit_medium_reproduces_the_unno_rachkovsky_solution():
    rng = np.random.default_rng(12)
    for trial in range(6):
        pol = rng.normal(size=3)
        pol *= rng.uniform(0.1, 0.5) / np.linalg.norm(pol)
        k6 = np.concatenate([pol, rng.normal(size=3) * 0.6])
        A = np.array([2.0, *rng.normal(size=3) * 0.2])
        Bp = np.array([0.05, *rng.normal(size=3) * 0.01])
        atm = explicit_slab(k6, A, Bp)
        p = oracle.Problem(atm, 1, 1, 2, 3, x_max=1.0)
        mu = np.array([1.0, 0.6, 0.35])
        chi = np.array([0.0, 1.1, 4.0])
        out = oracle.emergent(p, np.zeros(atm["chi"].shape + (6,)), mu, chi)
        M = np.eye(4) + _kprime(k6)
        Mi = np.linalg.inv(M)
        S_top = A + Bp * atm["z"][-1]
        for j, x in enumerate(np.linspace(-1.0, 1.0, 3)):
            eta = 10.0 * np.exp(-x * x)
            for d in range(3):
                exact = Mi @ S_top - Mi @ Mi @ Bp * mu[d] / eta
                got = out[d, j, 0, 0]
                assert np.allclose(got, exact, rtol=0, atol=1e-11 * np.abs(exact[0])), (trial, j, d, got, exact)
