"""Polarized multilevel atom on the GPU (porta_ml_* with polarized = 1) against
the oracle (oracle/mlpol.py): per-line radiation tensors J^K_Q (K = 0, 1, 2),
one update of the 69 multipoles per voxel from the same sums, iterations, the
converged solution and graph replay. The starting multipoles carry alignment
and orientation (K = 1, 2), so the dichroism (eta_Q, eta_U, eta_V) and the
orientation emission (eps_V) of every line are exercised.

Tolerances. FP64: 1e-10 relative on J^0_0, 1e-10 of J^0_0 on J^1_Q and J^2_Q, and one
update from the same sums to 1e-11 of the largest unknown (the two sides
assemble the same rate equations from differently ordered sums and solve them
by elimination with pivoting). FP32 sweeps: J^0_0 to 2e-5 relative and J^1_Q, J^2_Q to
2e-6 of J^0_0 (the two-level tolerances), populations after iterations and at
convergence to 1e-4 relative, multipole ratios rho^K_Q / rho^0_0 to 1e-5
absolute.
"""
import numpy as np
import pytest

import paper_1307_4217_gb300 as P
import synth
from oracle import ml, mlpol

pytestmark = pytest.mark.gpu

QUAD = (2, 4, 5)


def _case(nx=6, ny=5, nz=8, seed=2, eps_range=(1e-3, 1e-1)):
    atm = synth.multilevel_box(nx, ny, nz, seed=seed, tau_top=1e-3, tau_bot=1e2)
    # first-order Zeeman term within its validity at these fields (2 zeta |B| (x_max + |v|) < 1)
    atm["zeta"] = 5e-5
    atom = synth.multilevel_atom(seed=seed + 1, eps_range=eps_range)
    tab = mlpol.Tables(atom)
    x = mlpol.lte_unknowns(tab, atm["kT"])
    rng = np.random.default_rng(seed)
    rb = mlpol.real_basis(atom)
    for k, (i, K, Q, part) in enumerate(rb):
        r00 = x[..., rb.index((i, 0, 0, 0))]
        if K == 0:
            x[..., k] *= np.exp(0.2 * rng.normal(size=r00.shape))
        else:
            x[..., k] = 0.02 * r00 * rng.normal(size=r00.shape)
    return atm, atom, tab, x


def _ctx(atm, atom, prec, x):
    c = P.MlContext(atm, atom, *QUAD, precision=prec, polarized=True)
    c.set_atmosphere(atm)
    c.set_unknowns(x)
    return c


def _j9(jb):
    """GPU [line][grid][9] -> oracle [grid][line][9] (J00, J10, Re/Im J11, J20, Re/Im J21, Re/Im J22)"""
    return np.moveaxis(np.asarray(jb), 0, -2)


def _bvec(atm):
    return np.stack([atm["bx"], atm["by"], atm["bz"]], -1)


def test_sizes_and_unknown_layout():
    atm, atom, tab, x = _case()
    ctx = _ctx(atm, atom, P.PORTA_FP64, x)
    assert ctx.nunk == 69
    assert np.array_equal(ctx.get_unknowns(), x)
    pops = ctx.get_pops()
    assert np.allclose(pops, tab.populations(x), rtol=1e-15)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_line_radiation_tensors_match_oracle(prec):
    atm, atom, tab, x = _case()
    ctx = _ctx(atm, atom, prec, x)
    jb, ls = ctx.ml_formal_solve()
    oj, ol = mlpol.formal_solve_lines(atm, atom, tab, x, QUAD)
    gj = _j9(jb)
    fp64 = prec == P.PORTA_FP64
    j00 = oj[..., 0]
    assert np.max(np.abs(gj[..., 0] - j00) / j00) < (1e-10 if fp64 else 2e-5)
    assert np.max(np.abs(gj[..., 1:9] - oj[..., 1:9]) / j00[..., None]) < (1e-10 if fp64 else 2e-6)
    # orientation and Zeeman circular polarization give J^1_Q
    assert np.max(np.abs(oj[..., 1:4]) / j00[..., None]) > 1e-3
    assert np.max(np.abs(np.moveaxis(ls, 0, -1) - ol)) < (1e-10 if fp64 else 2e-5) * np.max(ol)


def test_update_matches_oracle_update():
    atm, atom, tab, x = _case(seed=4)
    ctx = _ctx(atm, atom, P.PORTA_FP64, x)
    jb, ls = ctx.ml_formal_solve()
    change = ctx.ml_see_update()
    got = ctx.get_unknowns()
    want, wchange = mlpol.see_update(tab, atm["kT"], x, _j9(jb), np.moveaxis(ls, 0, -1), _bvec(atm))
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))
    assert abs(change - wchange) < 1e-9 * wchange


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_iterations_match_oracle(prec):
    atm, atom, tab, x = _case(seed=5)
    ctx = _ctx(atm, atom, prec, x)
    ctx.ml_iterate(3)
    got = ctx.get_unknowns()
    want, _ = mlpol.iterate(atm, atom, tab, x, QUAD, 3)
    fp64 = prec == P.PORTA_FP64
    pg, pw = tab.populations(got), tab.populations(want)
    assert np.max(np.abs(pg / pw - 1)) < (1e-9 if fp64 else 1e-4)
    rb = mlpol.real_basis(atom)
    r00 = np.stack([want[..., rb.index((i, 0, 0, 0))] for (i, K, Q, p) in rb], -1)
    assert np.max(np.abs((got - want) / r00)) < (1e-9 if fp64 else 1e-5)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_converged_solution_matches_oracle(prec):
    atm, atom, tab, _ = _case(nx=4, ny=4, nz=8, seed=7, eps_range=(3e-2, 1e-1))
    x0 = mlpol.lte_unknowns(tab, atm["kT"])
    want = x0
    for _ in range(200):
        want, ch = mlpol.iterate(atm, atom, tab, want, QUAD, 1)
        if ch < 1e-12:
            break
    ctx = _ctx(atm, atom, prec, x0)
    for _ in range(30):
        ch = ctx.ml_iterate(10)
        if ch < (1e-12 if prec == P.PORTA_FP64 else 1e-7):
            break
    got = ctx.get_unknowns()
    rb = mlpol.real_basis(atom)
    r00 = np.stack([want[..., rb.index((i, 0, 0, 0))] for (i, K, Q, p) in rb], -1)
    fp64 = prec == P.PORTA_FP64
    assert np.max(np.abs(tab.populations(got) / tab.populations(want) - 1)) < (1e-9 if fp64 else 1e-4)
    assert np.max(np.abs((got - want) / r00)) < (1e-9 if fp64 else 1e-5)
    # atomic polarization is present (alignment of the upper levels)
    assert np.max(np.abs(want[..., rb.index((3, 2, 0, 0))] / want[..., rb.index((3, 0, 0, 0))])) > 1e-4


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_refined_solve_equals_fp64_elimination(prec):
    """The default solve of the K > 0 block (FP32 factors, FP64 refinement) against the
    FP64 elimination of the whole system, over iterations from oriented multipoles."""
    atm, atom, tab, x = _case(seed=11)
    a = _ctx(atm, atom, prec, x)
    b = _ctx(atm, atom, prec, x)
    b.set_solve(1)
    # FP32 sweeps: one iteration (afterwards the two unknowns, equal to ~1e-13, may round to
    # FP32 sources one ulp apart)
    n = 2 if prec == P.PORTA_FP64 else 1
    a.ml_iterate(n)
    b.ml_iterate(n)
    ga, gb = a.get_unknowns(), b.get_unknowns()
    assert np.max(np.abs(ga - gb)) < 1e-11 * np.max(np.abs(gb))
    with pytest.raises(P.PortaError):
        a.set_solve(2)


def test_graph_replay_equals_eager_iterations():
    import torch
    atm, atom, tab, x = _case(seed=6)
    a = _ctx(atm, atom, P.PORTA_FP32, x)
    b = _ctx(atm, atom, P.PORTA_FP32, x)
    s = torch.cuda.Stream()
    b.set_stream(s)
    a.ml_iterate(3)
    with torch.cuda.stream(s):
        b.run_iterations(3)
    s.synchronize()
    assert np.array_equal(a.get_unknowns(), b.get_unknowns())


def test_invalid_inputs_are_rejected():
    atm, atom, tab, x = _case()
    ctx = P.MlContext(atm, atom, *QUAD, precision=P.PORTA_FP32, polarized=True)
    no_field = {k: v for k, v in atm.items() if k not in ("bx", "by", "bz")}
    with pytest.raises(P.PortaError):
        ctx.set_atmosphere(no_field)
    ctx.set_atmosphere(atm)
    ctx.set_unknowns(x)
    with pytest.raises(P.PortaError):
        ctx.mg_setup(4)                          # 6 x 5 horizontal planes cannot be halved twice
    # a Zeeman splitting that makes |eta_V| > eta_I in the line wings is rejected
    strong = P.MlContext(atm, atom, *QUAD, precision=P.PORTA_FP32, polarized=True, zeta=3.5e-4)
    with pytest.raises(P.PortaError):
        strong.set_atmosphere(atm)


def _mg_case():
    atm = synth.multilevel_box(8, 8, 17, seed=2, tau_top=1e-2, tau_bot=1e2)
    atm["zeta"] = 5e-5
    atom = synth.multilevel_atom(seed=3, eps_range=(1e-2, 3e-2))
    return atm, atom, mlpol.Tables(atom)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_multigrid_cycle_matches_oracle(prec):
    quad = (2, 4, 5)
    atm, atom, tab = _mg_case()
    x0 = mlpol.lte_unknowns(tab, atm["kT"])
    ctx = P.MlContext(atm, atom, *quad, precision=prec, polarized=True)
    ctx.set_atmosphere(atm)
    ctx.set_unknowns(x0)
    ctx.mg_setup(3)
    assert ctx.mg_levels() == [(8, 8, 17), (4, 4, 9), (2, 2, 5)]
    ch = ctx.mg_vcycle(2, 4, 8)
    got = ctx.get_unknowns()
    want = mlpol.vcycle(ml.hierarchy(atm, 3), atom, tab, quad, x0)
    rb = mlpol.real_basis(atom)
    r00 = np.stack([want[..., rb.index((i, 0, 0, 0))] for (i, K, Q, p) in rb], -1)
    fp64 = prec == P.PORTA_FP64
    assert np.max(np.abs((got - want) / r00)) < (1e-9 if fp64 else 1e-4)
    pw, p0 = tab.populations(want), tab.populations(x0)
    wch = np.max(np.abs(pw - p0) / p0)
    assert abs(ch - wch) < (1e-8 if fp64 else 1e-3) * wch


def test_multigrid_reaches_the_jacobi_fixed_point():
    quad = (2, 4, 5)
    atm, atom, tab = _mg_case()
    x0 = mlpol.lte_unknowns(tab, atm["kT"])

    def make(x):
        c = P.MlContext(atm, atom, *quad, precision=P.PORTA_FP64, polarized=True)
        c.set_atmosphere(atm)
        c.set_unknowns(x)
        return c
    a = make(x0)
    a.mg_setup(3)
    for _ in range(9):
        ch = a.mg_vcycle(2, 4, 8)
    assert ch < 1e-9
    b = make(a.get_unknowns())
    assert b.ml_iterate(1) < 1e-9


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_emergent_line_profiles_match_oracle(prec):
    """Emergent Stokes profiles of every line (with the dichroism and emissivity
    of the current multipoles) against the oracle's emergent formal solution."""
    import oracle
    atm, atom, tab, x = _case(seed=9)
    ctx = _ctx(atm, atom, prec, x)
    mu, az = synth.emergent_directions()
    src = mlpol.line_source_multipoles(tab, x)
    for li in range(4):
        got = ctx.emergent_stokes(li, mu, az)
        want = oracle.emergent(mlpol.line_problem(atm, atom, tab, x, li, QUAD), src[..., li, :], mu, az)
        I = want[..., :1]
        if prec == P.PORTA_FP64:
            assert np.max(np.abs(got - want) / I) < 1e-10, li
        else:
            assert np.max(np.abs(got[..., 0] - want[..., 0]) / want[..., 0]) < 2e-5, li
            assert np.max(np.abs(got[..., 1:] - want[..., 1:]) / I) < 2e-6, li
        assert np.max(np.abs(want[..., 1:3]) / I) > 1e-5        # linear polarization present
