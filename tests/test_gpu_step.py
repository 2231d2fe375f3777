"""The GPU's BESSER-DELO step with a general propagation matrix (all seven
elements; Eq. 7 with kappa^-1 of Eq. 8) against the oracle's step, and against
the exact solution of the Unno-Rachkovsky problem: a constant propagation
matrix and a source vector linear in optical depth give a linear Stokes
vector, I = K~^-1 S0 - K~^-2 S1 + K~^-1 S1 s, which the step reproduces
exactly (to rounding) over a chain of steps. FP64: 1e-11 (the oracle's own
tolerance on this pin); FP32: 2e-5 relative to the chain's largest |I|."""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P

pytestmark = pytest.mark.gpu


def _row(IM, etaM, epsM, etaO, epsO, etaP_I, epsP, dsM, dsP, has_p):
    return np.concatenate([IM, etaM, epsM, etaO, epsO, [etaP_I], epsP, [dsM, dsP, 1.0 if has_p else 0.0]])


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-11), (P.PORTA_FP32, 2e-5)])
def test_general_step_matches_the_oracle_on_random_matrices(prec, tol):
    rng = np.random.default_rng(61)
    rows, want = [], []
    for _ in range(400):
        def eta():
            pol = rng.normal(size=3)
            pol *= rng.uniform(0.0, 0.95) / np.linalg.norm(pol)
            return np.array([rng.uniform(0.2, 3.0), *(pol * 1.0), *(rng.normal(size=3) * 0.8)]) * 1.0
        eM, eO = eta(), eta()
        eM[1:] *= eM[0]
        eO[1:] *= eO[0]
        IM = np.array([rng.uniform(0.5, 2), *rng.normal(size=3) * 0.1])
        sM, sO, sP = (np.array([rng.uniform(0.5, 2), *rng.normal(size=3) * 0.1]) for _ in range(3))
        etaP = rng.uniform(0.2, 3.0)
        dsM, dsP = 10 ** rng.uniform(-3, 0.7), 10 ** rng.uniform(-3, 0.7)
        has_p = bool(rng.integers(0, 5))
        epsM, epsO, epsP = sM * eM[0], sO * eO[0], sP * etaP
        rows.append(_row(IM, eM, epsM, eO, epsO, etaP, epsP, dsM, dsP, has_p))
        IO, ls = oracle.step(4, IM, eM, epsM, eO, epsO, etaP, epsP, dsM, dsP, has_p)
        want.append(np.concatenate([IO, [ls]]))
    rc, got = P.porta_eval_step(prec, np.array(rows))
    assert rc == P.PORTA_OK
    want = np.array(want)
    scale = np.abs(want[:, :1])
    assert np.max(np.abs(got[:, :4] - want[:, :4]) / scale) < tol
    assert np.max(np.abs(got[:, 4] - want[:, 4]) / want[:, 4]) < tol


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-11), (P.PORTA_FP32, 2e-5)])
def test_general_step_reproduces_the_unno_rachkovsky_solution(prec, tol):
    rng = np.random.default_rng(62)
    for trial in range(10):
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
        scale = max(np.abs(exact(s[0])).max(), np.abs(exact(s[-1])).max())
        for i in range(1, n):
            has_p = i + 1 < n
            Sp = S0 + S1 * s[i + 1] if has_p else np.zeros(4)
            row = _row(I, eta, S0 + S1 * s[i - 1], eta, S0 + S1 * s[i], 1.0, Sp, h, h, has_p)
            rc, out = P.porta_eval_step(prec, row[None])
            assert rc == P.PORTA_OK
            I = out[0, :4]
            assert np.max(np.abs(I - exact(s[i]))) < tol * scale, (trial, i, I, exact(s[i]))


def test_general_step_rejects_bad_inputs():
    row = _row(np.ones(4), [1, 0, 0, 0, 0, 0, 0], np.ones(4), [1, 0, 0, 0, 0, 0, 0], np.ones(4), 1.0, np.ones(4),
               0.1, 0.1, True)
    bad = row.copy()
    bad[4] = 0.0
    assert P.porta_eval_step(P.PORTA_FP64, bad[None])[0] == P.PORTA_EINVAL
    bad = row.copy()
    bad[0] = np.nan
    assert P.porta_eval_step(P.PORTA_FP32, bad[None])[0] == P.PORTA_EINVAL
