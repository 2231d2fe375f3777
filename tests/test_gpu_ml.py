"""Multilevel atom without polarization on the GPU (porta_ml_*) against the
oracle (oracle/ml.py): the per-line formal solutions and sums, the rate
equation update, iterations and the converged populations.

Tolerances. FP64: 1e-10 relative (the two sides differ only in summation
order). FP32 sweeps: Jbar to 2e-5 relative and Lambda-bar* to 2e-5 of its
largest value (the FP32 formal solution of the two-level tests); the update
itself runs in FP64, so one update from the same sums agrees to 1e-11; the
converged populations agree to 1e-4 relative.
"""
import numpy as np
import pytest

import paper_1307_4217_gb300 as P
import synth
from oracle import ml

pytestmark = pytest.mark.gpu

QUAD = (2, 4, 7)


def _case(nx=8, ny=6, nz=12, seed=2, eps_range=(1e-3, 1e-1)):
    atm = synth.multilevel_box(nx, ny, nz, seed=seed, tau_top=1e-3, tau_bot=1e2)
    atom = synth.multilevel_atom(seed=seed + 1, eps_range=eps_range)
    pops = ml.lte_populations(atom, atm["kT"])
    pops = pops * np.exp(0.2 * np.random.default_rng(seed).normal(size=pops.shape))
    return atm, atom, pops / pops.sum(-1, keepdims=True)


def _ctx(atm, atom, prec, pops):
    c = P.MlContext(atm, atom, *QUAD, precision=prec)
    c.set_atmosphere(atm)
    c.set_pops(pops)
    return c


def _lines(a):
    """[line][voxel] -> (nz, ny, nx, nline)"""
    return np.moveaxis(np.asarray(a), 0, -1)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_line_formal_solutions_match_oracle(prec):
    atm, atom, pops = _case()
    ctx = _ctx(atm, atom, prec, pops)
    jb, ls = ctx.ml_formal_solve()
    oj, ol = ml.formal_solve_lines(atm, atom, pops, QUAD)
    tol = 1e-10 if prec == P.PORTA_FP64 else 2e-5
    assert np.max(np.abs(_lines(jb) - oj) / oj) < tol
    assert np.max(np.abs(_lines(ls) - ol)) < tol * np.max(ol)


def test_update_matches_oracle_update():
    atm, atom, pops = _case(seed=4)
    ctx = _ctx(atm, atom, P.PORTA_FP32, pops)
    jb, ls = ctx.ml_formal_solve()
    change = ctx.ml_see_update()
    new = ctx.get_pops()
    want, wchange = ml.see_update(atom, atm["kT"], pops, _lines(jb), _lines(ls))
    assert np.max(np.abs(new / want - 1)) < 1e-11
    assert abs(change - wchange) <= 1e-11 * wchange


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_iterations_match_oracle(prec):
    atm, atom, pops = _case(seed=5)
    ctx = _ctx(atm, atom, prec, pops)
    ctx.ml_iterate(4)
    got = ctx.get_pops()
    want, _ = ml.iterate(atm, atom, pops, QUAD, 4)
    tol = 1e-10 if prec == P.PORTA_FP64 else 1e-4
    assert np.max(np.abs(got / want - 1)) < tol


def test_graph_replay_equals_eager_iterations():
    import torch
    atm, atom, pops = _case(seed=6)
    a = _ctx(atm, atom, P.PORTA_FP32, pops)
    b = _ctx(atm, atom, P.PORTA_FP32, pops)
    s = torch.cuda.Stream()
    b.set_stream(s)
    a.ml_iterate(3)
    with torch.cuda.stream(s):
        b.run_iterations(3)
    s.synchronize()
    assert np.array_equal(a.get_pops(), b.get_pops())


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_converged_populations_match_oracle(prec):
    atm, atom, pops0 = _case(nx=4, ny=4, nz=10, seed=7, eps_range=(3e-2, 1e-1))
    pops = ml.lte_populations(atom, atm["kT"])
    want = pops
    for _ in range(400):
        want, ch = ml.iterate(atm, atom, want, QUAD, 1)
        if ch < 1e-12:
            break
    ctx = _ctx(atm, atom, prec, pops)
    ch = 1.0
    for _ in range(40):
        ch = ctx.ml_iterate(10)
        if ch < (1e-12 if prec == P.PORTA_FP64 else 1e-7):
            break
    got = ctx.get_pops()
    tol = 1e-9 if prec == P.PORTA_FP64 else 1e-4
    assert np.max(np.abs(got / want - 1)) < tol
    assert np.max(np.abs(got / ml.lte_populations(atom, atm["kT"]) - 1)) > 1e-2


def test_autotuned_launch_gives_the_same_sums():
    atm, atom, pops = _case(nx=16, ny=16, nz=12, seed=8)
    a = _ctx(atm, atom, P.PORTA_FP32, pops)
    j0, l0 = a.ml_formal_solve()
    a.autotune()
    a.set_pops(pops)
    j1, l1 = a.ml_formal_solve()
    assert np.max(np.abs(j1 - j0) / j0) < 1e-6


def test_invalid_inputs_are_rejected():
    atm, atom, pops = _case()
    ctx = P.MlContext(atm, atom, *QUAD, precision=P.PORTA_FP32)
    with pytest.raises(P.PortaError):
        ctx.set_pops(pops)                     # atmosphere first
    ctx.set_atmosphere(atm)
    inv = pops.copy()
    inv[..., 3] = 10 * inv[..., 0]             # upper level above its lower level's weight: inversion
    with pytest.raises(P.PortaError):
        ctx.set_pops(inv)
    ctx.set_pops(pops)
    with pytest.raises(P.PortaError):
        ctx.set_rho(np.ones(ctx.grid_shape + (1,)))
    bad = dict(atom)
    bad["eps"] = np.array([0.5, 1.0, 0.5, 0.5])
    with pytest.raises(P.PortaError):
        P.MlContext(atm, bad, *QUAD)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_multigrid_cycles_match_oracle(prec):
    quad = (2, 4, 5)
    atm = synth.multilevel_box(8, 8, 17, seed=2, tau_top=1e-2, tau_bot=1e2)
    atom = synth.multilevel_atom(seed=3, eps_range=(1e-2, 3e-2))
    p0 = ml.lte_populations(atom, atm["kT"])
    levels = ml.hierarchy(atm, 3)
    ctx = P.MlContext(atm, atom, *quad, precision=prec)
    ctx.set_atmosphere(atm)
    ctx.set_pops(p0)
    ctx.mg_setup(3)
    assert ctx.mg_levels() == [(8, 8, 17), (4, 4, 9), (2, 2, 5)]
    want = p0
    tol = 1e-9 if prec == P.PORTA_FP64 else 1e-4
    for _ in range(2):
        prev = want
        want = ml.vcycle(levels, atom, quad, want)
        ch = ctx.mg_vcycle(2, 4, 8)
        got = ctx.get_pops()
        assert np.max(np.abs(got / want - 1)) < tol
        wch = np.max(np.abs(want - prev) / prev)
        assert abs(ch - wch) < 10 * tol * wch


def test_multigrid_reaches_the_jacobi_fixed_point():
    quad = (2, 4, 5)
    atm = synth.multilevel_box(8, 8, 17, seed=4, tau_top=1e-2, tau_bot=1e2)
    atom = synth.multilevel_atom(seed=5, eps_range=(1e-2, 3e-2))
    p0 = ml.lte_populations(atom, atm["kT"])
    def make(pops):
        c = P.MlContext(atm, atom, *quad, precision=P.PORTA_FP64)
        c.set_atmosphere(atm)
        c.set_pops(pops)
        return c
    a = make(p0)
    a.mg_setup(3)
    for _ in range(8):
        ch = a.mg_vcycle(2, 4, 8)
    assert ch < 1e-9
    b = make(a.get_pops())
    # a Jacobi iteration leaves the multigrid solution in place
    assert b.ml_iterate(1) < 1e-9


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_emergent_line_profiles_match_oracle(prec):
    import oracle
    atm, atom, pops = _case(seed=10)
    ctx = _ctx(atm, atom, prec, pops)
    mu, az = synth.emergent_directions()
    S = ml.source_function(atom, pops)
    for k in range(4):
        got = ctx.emergent_stokes(k, mu, az)
        want = oracle.emergent(ml.line_problem(atm, atom, pops, k, QUAD), S[..., k:k + 1], mu, az)
        assert np.max(np.abs(got - want) / want) < (1e-10 if prec == P.PORTA_FP64 else 2e-5), k
