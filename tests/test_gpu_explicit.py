"""The emergent sweep with a general propagation matrix on the GPU (all seven
elements of Eqs. 7-8: porta_set_explicit_medium) against the exact
Unno-Rachkovsky solution of a thick slab with constant K' and a source linear
in height, and against the oracle's sweep on a box whose K' and S vary between
voxels; the J^K_Q formal solution over that box against the oracle's. FP64 1e-10, FP32 1e-5 (the parity tolerances of the two-level sweeps)."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
from test_oracle_explicit import _kprime, explicit_slab

pytestmark = pytest.mark.gpu


def _ctx(atm, prec):
    ctx = P.Context(atm, 1, 1, 2, 3, x_max=1.0, precision=prec)
    ctx.set_atmosphere(atm)
    rho = np.zeros(atm["chi"].shape + (6,))
    rho[..., 0] = 1.0                    # the unknowns are not used by an explicit medium
    ctx.set_rho(rho)
    ctx.set_explicit_medium(atm["kexpl"], atm["sexpl"])
    return ctx


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_explicit_slab_gives_the_unno_rachkovsky_solution(prec, tol):
    rng = np.random.default_rng(21)
    for trial in range(4):
        pol = rng.normal(size=3)
        pol *= rng.uniform(0.1, 0.5) / np.linalg.norm(pol)
        k6 = np.concatenate([pol, rng.normal(size=3) * 0.6])
        A = np.array([2.0, *rng.normal(size=3) * 0.2])
        Bp = np.array([0.05, *rng.normal(size=3) * 0.01])
        atm = explicit_slab(k6, A, Bp)
        ctx = _ctx(atm, prec)
        mu = np.array([1.0, 0.6, 0.35])
        chi = np.array([0.0, 1.1, 4.0])
        out = ctx.emergent_stokes(mu, chi)
        ctx.close()
        Mi = np.linalg.inv(np.eye(4) + _kprime(k6))
        S_top = A + Bp * atm["z"][-1]
        for j, x in enumerate(np.linspace(-1.0, 1.0, 3)):
            eta = 10.0 * np.exp(-x * x)
            for d in range(3):
                exact = Mi @ S_top - Mi @ Mi @ Bp * mu[d] / eta
                assert np.max(np.abs(out[d, j] - exact)) < tol * abs(exact[0]), (trial, j, d)


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_explicit_medium_matches_the_oracle_on_a_varying_box(prec, tol):
    rng = np.random.default_rng(22)
    nx, ny, nz = 6, 8, 12
    atm = explicit_slab(np.zeros(6), np.array([1.0, 0, 0, 0]), np.zeros(4), nx=nx, ny=ny, nz=nz, chi=2.0, dz=0.5)
    shape = (nz, ny, nx)
    atm["chi"] = 2.0 * np.exp(0.2 * rng.normal(size=shape))
    atm["vel"] = 0.3 * rng.normal(size=shape)
    k = rng.normal(size=(6,) + shape) * 0.15
    atm["kexpl"] = k
    s = np.empty((4,) + shape)
    s[0] = rng.uniform(0.5, 1.5, shape)
    s[1:] = rng.normal(size=(3,) + shape) * 0.05
    atm["sexpl"] = s
    ctx = _ctx(atm, prec)
    mu = np.array([1.0, 0.45, 0.8])
    chi = np.array([0.0, 0.7, 3.9])
    got = ctx.emergent_stokes(mu, chi)
    ctx.close()
    want = oracle.emergent(oracle.Problem(atm, 1, 1, 2, 3, x_max=1.0), np.zeros(shape + (6,)), mu, chi)
    assert np.max(np.abs(got - want) / np.abs(want[..., :1])) < tol


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_explicit_medium_radiation_tensors_match_the_oracle(prec, tol):
    """J^K_Q and Lambda-bar* of a formal solution over the varying explicit medium (the
    seven-element step in the global-memory sweep) against the oracle's."""
    rng = np.random.default_rng(23)
    nx, ny, nz = 6, 8, 12
    atm = explicit_slab(np.zeros(6), np.array([1.0, 0, 0, 0]), np.zeros(4), nx=nx, ny=ny, nz=nz, chi=2.0, dz=0.5)
    shape = (nz, ny, nx)
    atm["chi"] = 2.0 * np.exp(0.2 * rng.normal(size=shape))
    atm["vel"] = 0.3 * rng.normal(size=shape)
    atm["kexpl"] = rng.normal(size=(6,) + shape) * 0.15
    s = np.empty((4,) + shape)
    s[0] = rng.uniform(0.5, 1.5, shape)
    s[1:] = rng.normal(size=(3,) + shape) * 0.05
    atm["sexpl"] = s
    ctx = _ctx(atm, prec)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    ctx.close()
    jo, lo = oracle.formal_solve(oracle.Problem(atm, 1, 1, 2, 3, x_max=1.0), np.zeros(shape + (6,)))
    assert np.max(np.abs(jg - jo) / np.abs(jo[..., :1])) < tol
    assert np.max(np.abs(lg - lo) / np.abs(lo)) < tol
    # the magneto-optical and dichroic terms matter: without them the sums differ
    a0 = dict(atm)
    a0["kexpl"] = np.zeros_like(atm["kexpl"])
    j0, _ = oracle.formal_solve(oracle.Problem(a0, 1, 1, 2, 3, x_max=1.0), np.zeros(shape + (6,)))
    assert np.max(np.abs(j0 - jo) / np.abs(jo[..., :1])) > 100 * tol


def test_explicit_medium_errors_and_clearing():
    atm = explicit_slab(np.zeros(6), np.array([1.0, 0, 0, 0]), np.zeros(4), nz=8)
    ctx = _ctx(atm, P.PORTA_FP64)
    ctx.formal_solve()                   # the J^K_Q formal solution runs over the medium
    with pytest.raises(P.PortaError) as e:
        ctx.set_interpolation(2)
    assert e.value.code == P.PORTA_EINVAL
    ctx.set_explicit_medium(None, None)
    ctx.set_rho(np.concatenate([np.ones(atm["chi"].shape + (1,)), np.zeros(atm["chi"].shape + (5,))], -1))
    ctx.formal_solve()
    ctx.close()
