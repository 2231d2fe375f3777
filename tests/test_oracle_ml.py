"""Pins of the multilevel (unpolarized) oracle, oracle/ml.py: closed forms of
the thermal limit, the fixed point under Planckian radiation, conservation,
the reduction to the pinned two-level update, and the fixed point of the
preconditioned iteration against the plain rate equations."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ml


def _atom(eps_range=(1e-4, 1e-2), seed=0):
    return synth.multilevel_atom(seed=seed, eps_range=eps_range)


def _kT(shape, seed=1):
    return 0.5 * np.exp(0.05 * np.random.default_rng(seed).normal(size=shape))


def test_strong_collisions_give_boltzmann_populations():
    atom = _atom()
    atom["eps"] = np.full(4, 1.0 - 1e-11)
    kT = _kT((3, 4))
    rng = np.random.default_rng(2)
    pops = ml.lte_populations(atom, kT) * rng.uniform(0.5, 1.5, size=(3, 4, 5))
    pops /= pops.sum(-1, keepdims=True)
    jbar = rng.uniform(0.0, 2.0, size=(3, 4, 4)) * ml.planck(atom, kT)
    lstar = rng.uniform(0.0, 0.9, size=(3, 4, 4))
    new, _ = ml.see_update(atom, kT, pops, jbar, lstar)
    # n_i / n_0 = g_i exp(-E_i / kT) / g_0 (Boltzmann)
    g = 2.0 * atom["J"] + 1
    want = g * np.exp(-atom["E"] / kT[..., None])
    want /= want.sum(-1, keepdims=True)
    assert np.max(np.abs(new / want - 1)) < 1e-8


def test_lte_source_function_is_the_planck_function():
    atom = _atom()
    kT = _kT((5,))
    pops = ml.lte_populations(atom, kT)
    S = ml.source_function(atom, pops)
    # B = r^3 / (exp(dE/kT) - 1) with r = dE / dE_ref, written from the energies
    u, l = atom["lines"][:, 0], atom["lines"][:, 1]
    dE = atom["E"][u] - atom["E"][l]
    B = (dE / dE[0]) ** 3 / (np.exp(dE / kT[:, None]) - 1.0)
    assert np.allclose(S, B, rtol=1e-12, atol=0)
    assert np.allclose(ml.planck(atom, kT), B, rtol=1e-12, atol=0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_planckian_radiation_is_a_fixed_point(seed):
    atom = _atom(seed=seed)
    kT = _kT((2, 3, 4), seed=seed + 5)
    pops = ml.lte_populations(atom, kT)
    jbar = ml.planck(atom, kT)
    lstar = np.random.default_rng(seed).uniform(0.0, 0.99, size=jbar.shape)
    new, change = ml.see_update(atom, kT, pops, jbar, lstar)
    assert change < 1e-12


def test_rate_matrix_conserves_atoms():
    atom = _atom()
    kT = _kT((7,))
    rng = np.random.default_rng(3)
    M = ml.rate_matrix(atom, kT, rng.normal(size=(7, 4)), rng.uniform(size=(7, 4)))
    assert np.max(np.abs(M.sum(-2))) < 1e-6 * np.max(np.abs(M))
    pops = rng.uniform(0.1, 1, size=(7, 5))
    pops /= pops.sum(-1, keepdims=True)
    new, _ = ml.see_update(atom, kT, pops, rng.uniform(size=(7, 4)), rng.uniform(0, 0.5, size=(7, 4)))
    assert np.allclose(new.sum(-1), 1.0, rtol=0, atol=1e-14)


def test_two_level_atom_reduces_to_the_two_level_update():
    """Populations of a J = 0 -> 1 atom after one update give the source
    function of the pinned two-level update with eps' = C'/(A + C'),
    C' = C_ul (1 - exp(-dE/kT)), and B the line's Planck function."""
    atom = dict(J=np.array([0, 1]), E=np.array([0.0, 3.1]), lines=np.array([[1, 0]]),
                A=np.array([3e7]), eps=np.array([2e-3]))
    atm = synth.plane_parallel_box(3, 2, 4)
    shape = atm["chi"].shape
    rng = np.random.default_rng(4)
    kT = _kT(shape, seed=6)
    pops = ml.lte_populations(atom, kT) * np.stack([np.ones(shape), rng.uniform(0.5, 3, size=shape)], -1)
    pops /= pops.sum(-1, keepdims=True)
    jbar = rng.uniform(0.2, 1.5, size=shape + (1,)) * ml.planck(atom, kT)
    lstar = rng.uniform(0.0, 0.95, size=shape + (1,))
    new, _ = ml.see_update(atom, kT, pops, jbar, lstar)

    cul, _ = ml.collision_rates(atom, kT)
    cp = cul[0] * (1.0 - np.exp(-3.1 / kT))
    a2 = dict(atm)
    a2["eps"] = cp / (atom["A"][0] + cp)
    a2["bpl"] = ml.planck(atom, kT)[..., 0]
    p = oracle.Problem(a2, 0, 1, 1, 3)
    S_old = ml.source_function(atom, pops)
    S_two, _ = oracle.see_update(p, jbar, lstar[..., 0], S_old)
    assert np.allclose(ml.source_function(atom, new), S_two, rtol=1e-11, atol=0)


def test_converged_populations_solve_the_plain_rate_equations():
    """At the fixed point of the preconditioned iteration the populations solve
    the rate equations with the radiation field of their own formal solution."""
    atm = synth.multilevel_box(4, 4, 10, seed=2, tau_top=1e-2, tau_bot=1e2)
    atom = _atom(eps_range=(3e-2, 1e-1), seed=3)
    quad = (2, 4, 5)
    pops = ml.lte_populations(atom, atm["kT"])
    change = 1.0
    for _ in range(300):
        pops, change = ml.iterate(atm, atom, pops, quad, 1)
        if change < 1e-11:
            break
    assert change < 1e-11
    jbar, _ = ml.formal_solve_lines(atm, atom, pops, quad)
    plain = ml.solve_populations(ml.rate_matrix(atom, atm["kT"], jbar, np.zeros_like(jbar)))
    assert np.max(np.abs(plain / pops - 1)) < 1e-8
    # not LTE: the lines are out of equilibrium at the top
    assert np.max(np.abs(pops / ml.lte_populations(atom, atm["kT"]) - 1)) > 1e-2


def test_emissivity_follows_the_upper_population_alone():
    """chi_ul S_ul is the spontaneous emission: proportional to n_u and
    independent of n_l (stimulated emission cancels between the opacity and the
    source function); with n_u = 0 the opacity is chi s_ul n_l."""
    atom = _atom()
    rng = np.random.default_rng(8)
    chi = rng.uniform(0.5, 2.0, size=6)
    pops = rng.uniform(0.05, 0.3, size=(6, 5))
    e0 = ml.line_opacity(atom, chi, pops) * ml.source_function(atom, pops)
    p2 = pops.copy()
    p2[:, :3] *= 1.7                       # lower levels only
    assert np.allclose(ml.line_opacity(atom, chi, p2) * ml.source_function(atom, p2), e0, rtol=1e-12)
    p3 = pops.copy()
    p3[:, 3:] *= 0.25                      # upper levels only
    assert np.allclose(ml.line_opacity(atom, chi, p3) * ml.source_function(atom, p3), 0.25 * e0, rtol=1e-12)
    p4 = pops.copy()
    p4[:, 3:] = 0.0
    _, _, _, s = ml.line_tables(atom)
    lower = atom["lines"][:, 1]
    assert np.allclose(ml.line_opacity(atom, chi, p4), chi[:, None] * s * pops[:, lower], rtol=1e-14)


def test_update_with_the_unit_right_hand_side_is_the_update():
    atom = _atom()
    kT = _kT((3, 5))
    rng = np.random.default_rng(9)
    pops = ml.lte_populations(atom, kT) * rng.uniform(0.7, 1.3, size=(3, 5, 5))
    jbar = rng.uniform(0.5, 1.5, size=(3, 5, 4)) * ml.planck(atom, kT)
    lstar = rng.uniform(0, 0.9, size=(3, 5, 4))
    a, _ = ml.see_update(atom, kT, pops, jbar, lstar)
    b, _ = ml.see_update(atom, kT, pops, jbar, lstar, ml.f_fine((3, 5), 5))
    assert np.allclose(a, b, rtol=1e-14, atol=0)


def test_multigrid_cycles_reach_the_fixed_point_faster_than_jacobi():
    """Three V-cycles (2 pre, 4 post, 8 coarsest; three levels 8x8x17 -> 4x4x9
    -> 2x2x5) leave a residual f - A(n) over 30x below that of Jacobi at equal
    fine-grid cost (7 formal solutions per cycle); eight cycles reach a solution
    of the plain rate equations, which a further cycle leaves unchanged."""
    quad = (2, 4, 5)
    atm = synth.multilevel_box(8, 8, 17, seed=2, tau_top=1e-2, tau_bot=1e2)
    atom = _atom(eps_range=(1e-2, 3e-2), seed=3)
    p0 = ml.lte_populations(atom, atm["kT"])
    levels = ml.hierarchy(atm, 3)
    assert [lv.shape for lv in levels] == [(17, 8, 8), (9, 4, 4), (5, 2, 2)]
    f = ml.f_fine(p0.shape[:-1], 5)

    def res(x):
        return np.max(np.abs(f - ml.apply_A(atm, atom, x, quad)))
    p, q = p0.copy(), p0.copy()
    for _ in range(3):
        p = ml.vcycle(levels, atom, quad, p)
        q, _ = ml.iterate(atm, atom, q, quad, 7)
    assert res(p) * 30 < res(q)
    for _ in range(5):
        p = ml.vcycle(levels, atom, quad, p)
    jbar, _ = ml.formal_solve_lines(atm, atom, p, quad)
    plain = ml.solve_populations(ml.rate_matrix(atom, atm["kT"], jbar, np.zeros_like(jbar)))
    assert np.max(np.abs(plain / p - 1)) < 1e-9
    p2 = ml.vcycle(levels, atom, quad, p)
    assert np.max(np.abs(p2 / p - 1)) < 1e-10
