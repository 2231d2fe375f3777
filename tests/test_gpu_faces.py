"""Short characteristics ending on the first cell face they cross (Sec. 3.1,
porta_set_sc_faces(1), faces.cu) against the oracle's face sweep (oracle
`sc_faces=1`): J^K_Q and Lambda-bar* of a formal solution of a random box whose
grazing rays meet vertical faces (each such plane solved jointly, the periodic
chains closed), the Jacobi update from them, emergent Stokes profiles of
grazing lines of sight, graph replay, determinism, and the rejected
combinations. Tolerances as the bilinear parity tests: FP64 1e-10, FP32 1e-5
(the FP32 plane solve stops at 2e-7 of the plane's largest change)."""
import math

import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import initial_rho, make_ctx

pytestmark = pytest.mark.gpu


def _max_offset(atm, p):
    mu, chi, _ = oracle.rays(p)
    dz = np.min(np.abs(np.diff(atm["z"])))
    dx, dy = atm["lx"] / atm["nx"], atm["ly"] / atm["ny"]
    t = np.sqrt(1 - mu ** 2) / np.abs(mu)
    return np.max(dz * t * np.maximum(np.abs(np.cos(chi)) / dx, np.abs(np.sin(chi)) / dy))


def _check(jg, lg, jo, lo, tol):
    s = np.abs(jo[..., :1])
    assert np.max(np.abs(jg - jo) / s) < tol
    assert np.max(np.abs(lg - lo) / np.abs(lo)) < tol


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
@pytest.mark.parametrize("model", [0, 1])
def test_face_formal_solution_matches_oracle(prec, tol, model):
    atm = synth.random_box(9, 7, 10, seed=21, sigma_lnchi=0.1, sigma_v=0.3)
    rho = initial_rho(atm, model, seed=22)
    quad = (2, 4, 5)
    p = oracle.Problem(atm, model, *quad, sc_faces=1)
    assert _max_offset(atm, p) > 2.0              # grazing rays cross vertical faces
    ctx = make_ctx(atm, model, *quad, prec, rho=rho)
    ctx.set_sc_faces(1)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    jo, lo = oracle.formal_solve(p, rho)
    _check(jg, lg, jo, lo, tol)
    # the placement matters: the plane sweep gives another field
    jb, _ = oracle.formal_solve(oracle.Problem(atm, model, *quad), rho)
    assert np.max(np.abs(jb - jo) / np.abs(jo[..., :1])) > 100 * tol
    # the update from these sums is the oracle's
    ch = ctx.see_update()
    _, cho = oracle.see_update(p, jo, lo, rho)
    assert abs(ch - cho) < 10 * tol * cho
    ctx.close()


def test_face_formal_solution_is_deterministic_and_options_are_checked():
    atm = synth.random_box(8, 6, 8, seed=5)
    rho = initial_rho(atm, 1, seed=6)
    ctx = make_ctx(atm, 1, 2, 4, 3, P.PORTA_FP32, rho=rho)
    ctx.set_sc_faces(1)
    ctx.formal_solve()
    j1, l1 = ctx.accumulate_jkq()
    ctx.formal_solve()
    j2, l2 = ctx.accumulate_jkq()
    assert np.array_equal(j1, j2) and np.array_equal(l1, l2)
    with pytest.raises(P.PortaError):
        ctx.set_sc_faces(2)
    with pytest.raises(P.PortaError):
        ctx.set_interpolation(2)
    mu, az = synth.emergent_directions()
    with pytest.raises(P.PortaError):
        ctx.emergent_vjp(mu, az, np.ones((len(mu), 3, 6, 8, 4)))
    ctx.set_sc_faces(0)                          # back to the plane sweep
    ctx.formal_solve()
    j3, _ = ctx.accumulate_jkq()
    assert not np.array_equal(j1, j3)
    ctx.close()


def test_face_iterations_graph_replay_equals_eager():
    """Jacobi iterations with the face sweep captured as a CUDA graph (its work planes
    allocated before the capture) give the eager iterations' unknowns bitwise."""
    import torch
    atm = synth.random_box(8, 6, 8, seed=7)
    rho = initial_rho(atm, 1, seed=8)
    a = make_ctx(atm, 1, 2, 4, 3, P.PORTA_FP32, rho=rho)
    b = make_ctx(atm, 1, 2, 4, 3, P.PORTA_FP32, rho=rho)
    a.set_sc_faces(1)
    b.set_sc_faces(1)
    for _ in range(2):
        a.formal_solve()
        a.accumulate_jkq()
        a.see_update()
    s = torch.cuda.Stream()
    b.set_stream(s)
    with torch.cuda.stream(s):
        b.run_iterations(2)
    s.synchronize()
    assert np.array_equal(a.get_rho(), b.get_rho())
    a.close()
    b.close()


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_face_emergent_profiles_match_oracle(prec, tol):
    atm = synth.random_box(9, 7, 10, seed=23, sigma_lnchi=0.1, sigma_v=0.3)
    rho = initial_rho(atm, 1, seed=24)
    ctx = make_ctx(atm, 1, 2, 4, 5, prec, rho=rho)
    ctx.set_sc_faces(1)
    mu = np.array([1.0, 0.5, 0.2, 0.08])          # the last two meet vertical faces
    chi = np.array([0.0, 0.7, 2.2, 4.0])
    eg = ctx.emergent_stokes(mu, chi)
    p = oracle.Problem(atm, 1, 2, 4, 5, sc_faces=1)
    eo = oracle.emergent(p, rho, mu, chi)
    assert np.max(np.abs(eg - eo) / np.abs(eo[..., :1])) < tol
    # grazing lines of sight differ from the plane placement, the vertical one does not
    ep = oracle.emergent(oracle.Problem(atm, 1, 2, 4, 5), rho, mu, chi)
    assert np.max(np.abs(ep[0] - eo[0]) / np.abs(eo[0, ..., :1])) < 1e-12
    assert np.max(np.abs(ep[3] - eo[3]) / np.abs(eo[3, ..., :1])) > 100 * tol
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 2e-5)])
def test_multilevel_lines_with_face_intersections_match_oracle(prec, tol):
    """The line boxes of the multilevel atom through the face sweep (one launch over
    (line, ray, frequency group) items) against the oracle's per-line face sweeps;
    tolerances of the multilevel parity tests."""
    from oracle import ml
    atm = synth.multilevel_box(8, 6, 12, seed=2, tau_top=1e-3, tau_bot=1e2)
    atom = synth.multilevel_atom(seed=3, eps_range=(1e-3, 1e-1))
    pops = ml.lte_populations(atom, atm["kT"])
    quad = (2, 4, 7)
    assert _max_offset(atm, ml.line_problem(atm, atom, pops, 0, quad, sc_faces=1)) > 2.0
    c = P.MlContext(atm, atom, *quad, precision=prec)
    c.set_atmosphere(atm)
    c.set_pops(pops)
    c.set_sc_faces(1)
    jb, ls = c.ml_formal_solve()
    jb, ls = np.moveaxis(np.asarray(jb), 0, -1), np.moveaxis(np.asarray(ls), 0, -1)
    oj, ol = ml.formal_solve_lines(atm, atom, pops, quad, sc_faces=1)
    assert np.max(np.abs(jb - oj) / oj) < tol
    assert np.max(np.abs(ls - ol)) < tol * np.max(ol)
    pj, _ = ml.formal_solve_lines(atm, atom, pops, quad)
    assert np.max(np.abs(pj - oj) / oj) > 100 * tol
    c.close()


@pytest.mark.parametrize("prec,tol", [(P.PORTA_FP64, 1e-10), (P.PORTA_FP32, 1e-5)])
def test_batched_boxes_with_face_intersections_match_oracle(prec, tol):
    """Independent boxes of uneven size (their own cell sizes) in one face-sweep
    launch, box by box against the oracle's face sweep."""
    dims = [(9, 7, 10), (5, 12, 9), (12, 5, 6), (3, 3, 12)]
    atms = [synth.random_box(nx, ny, nz, seed=[60, b], sigma_lnchi=0.1, sigma_v=0.3)
            for b, (nx, ny, nz) in enumerate(dims)]
    rhos = [initial_rho(a, 1, seed=70 + b).reshape(-1, 6) for b, a in enumerate(atms)]
    ctx = P.BatchContext(atms, 1, 2, 4, 5, precision=prec)
    ctx.set_atmosphere(atms)
    ctx.set_rho(np.concatenate(rhos))
    ctx.set_sc_faces(1)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    grazing = 0
    for b, (atm, jb, lb) in enumerate(zip(atms, ctx.split(jg), ctx.split(lg))):
        p = oracle.Problem(atm, 1, 2, 4, 5, sc_faces=1)
        grazing += _max_offset(atm, p) > 2.0
        jo, lo = oracle.formal_solve(p, rhos[b].reshape(p.shape + (6,)))
        _check(jb, lb, jo.reshape(-1, 6), lo.ravel(), tol)
    assert grazing >= 2
    ctx.close()


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_polarized_multilevel_lines_with_face_intersections_match_oracle(prec):
    """The polarized multilevel lines (dichroism D^2_Q, orientation D^1_Q and S^1_Q,
    J^1_Q from Stokes V) through the face sweep against the oracle's per-line face
    sweeps; tolerances of the polarized multilevel parity tests."""
    from oracle import mlpol
    atm = synth.multilevel_box(6, 5, 8, seed=2, tau_top=1e-3, tau_bot=1e2)
    atm["zeta"] = 5e-5
    atom = synth.multilevel_atom(seed=3, eps_range=(1e-3, 1e-1))
    tab = mlpol.Tables(atom)
    x = mlpol.lte_unknowns(tab, atm["kT"])
    rng = np.random.default_rng(2)
    rb = mlpol.real_basis(atom)
    for k, (i, K, Q, part) in enumerate(rb):
        r00 = x[..., rb.index((i, 0, 0, 0))]
        if K == 0:
            x[..., k] *= np.exp(0.2 * rng.normal(size=r00.shape))
        else:
            x[..., k] = 0.02 * r00 * rng.normal(size=r00.shape)
    quad = (2, 4, 5)
    assert _max_offset(atm, mlpol.line_problem(atm, atom, tab, x, 0, quad, sc_faces=1)) > 2.0
    c = P.MlContext(atm, atom, *quad, precision=prec, polarized=True)
    c.set_atmosphere(atm)
    c.set_unknowns(x)
    c.set_sc_faces(1)
    jb, ls = c.ml_formal_solve()
    oj, ol = mlpol.formal_solve_lines(atm, atom, tab, x, quad, sc_faces=1)
    gj = np.moveaxis(np.asarray(jb), 0, -2)
    fp64 = prec == P.PORTA_FP64
    j00 = oj[..., 0]
    assert np.max(np.abs(gj[..., 0] - j00) / j00) < (1e-10 if fp64 else 2e-5)
    assert np.max(np.abs(gj[..., 1:9] - oj[..., 1:9]) / j00[..., None]) < (1e-10 if fp64 else 2e-6)
    assert np.max(np.abs(oj[..., 1:4]) / j00[..., None]) > 1e-3
    assert np.max(np.abs(np.moveaxis(ls, 0, -1) - ol)) < (1e-10 if fp64 else 2e-5) * np.max(ol)
    pj, _ = mlpol.formal_solve_lines(atm, atom, tab, x, quad)
    assert np.max(np.abs(pj[..., 0] - j00) / j00) > 1e-6
    c.close()
