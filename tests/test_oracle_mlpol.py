"""Pins of the polarized multilevel oracle (oracle/mlpol.py): conservation of
atoms, hermiticity, the reduction to the pinned unpolarized multilevel update
and to the pinned two-level polarized atom (with the Hanle effect), dark
states of the dipole selection rules, the LTE fixed point, and the fixed point
of the preconditioned iteration."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ml, mlpol
from oracle.wigner import w3j


def _atom2(Jl, Ju, A=3e7, eps=2e-3, dE=3.1):
    return dict(J=np.array([Jl, Ju]), E=np.array([0.0, dE]), lines=np.array([[1, 0]]), A=np.array([A]),
                eps=np.array([eps]))


def _sublevels(tab, level, p):
    """real unknowns of a level whose sublevels M = -J..J carry populations p (no coherences):
    rho^K_0 = sum_M (-1)^(J-M) sqrt(2K+1) (J J K; M -M 0) p_M"""
    J = tab.J[level]
    x = np.zeros(len(tab.rows))
    rb = mlpol.real_basis(tab.atom)
    Ms = np.arange(-J, J + 1)
    for K in range(int(round(2 * J)) + 1):
        v = sum((-1) ** int(round(J - M)) * np.sqrt(2 * K + 1) * w3j(J, J, K, M, -M, 0) * pm for M, pm in zip(Ms, p))
        x[rb.index((level, K, 0, 0))] = v
    return x


def _beam(mu, chi, stokes):
    """radiation tensors (real layout, Kr = 0, 1, 2) of a beam of Stokes (I, Q, U) along (mu, chi)"""
    t = oracle.tkq(mu, chi)              # rows I, Q, U; (T00, T20, Re T21, Im T21, Re T22, Im T22)
    j6 = sum(stokes[i] * t[i] for i in range(3))
    out = np.zeros(9)
    out[0] = j6[0]
    out[4:9] = j6[1:6]
    return out


def test_rate_equations_conserve_atoms_and_hermiticity():
    atom = synth.multilevel_atom(seed=0)
    for stim in (False, True):
        tab = mlpol.Tables(atom, stimulated=stim)
        assert tab.n == 69 and len(tab.rows) == 69
        rng = np.random.default_rng(1)
        jb = rng.normal(size=(1, 4, 9))
        jb[..., 0] = np.abs(jb[..., 0]) + 1
        Mc = tab.matrix(np.array([0.5]), jb, rng.normal(size=(1, 3)) * 10)
        R = tab.real_system(Mc)[0]
        # d/dt sum_J sqrt(2J+1) rho^0_0(J) = 0 for every state
        assert np.max(np.abs(tab.trace @ R)) < 1e-12 * np.max(np.abs(R))
        xc = tab.to_complex(rng.normal(size=69))
        y = Mc[0] @ xc
        for k, (i, K, Q) in enumerate(tab.cb):
            kk = tab.idx[(i, K, -Q)]
            assert abs(y[kk] - (-1) ** Q * np.conj(y[k])) < 1e-12 * np.max(np.abs(y))


def test_unpolarized_radiation_reduces_to_the_population_update():
    atom = synth.multilevel_atom(seed=2)
    tab = mlpol.Tables(atom)
    rng = np.random.default_rng(3)
    kT = np.array([0.5, 0.45, 0.52])
    pops = ml.lte_populations(atom, kT) * rng.uniform(0.6, 1.4, size=(3, 5))
    pops /= pops.sum(-1, keepdims=True)
    x0 = np.zeros((3, 69))
    rb = mlpol.real_basis(atom)
    for i in range(5):
        x0[:, rb.index((i, 0, 0, 0))] = pops[:, i] / np.sqrt(tab.g[i])
    jb = np.zeros((3, 4, 9))
    jb[..., 0] = rng.uniform(0.3, 1.5, size=(3, 4)) * ml.planck(atom, kT)
    ls = rng.uniform(0, 0.9, size=(3, 4))
    new, _ = mlpol.see_update(tab, kT, x0, jb, ls, np.zeros((3, 3)))
    want, _ = ml.see_update(atom, kT, pops, jb[..., 0], ls)
    assert np.max(np.abs(tab.populations(new) / want - 1)) < 1e-11
    pol = np.delete(new, [rb.index((i, 0, 0, 0)) for i in range(5)], axis=-1)
    assert np.max(np.abs(pol)) < 1e-14


def test_two_level_atom_reduces_to_the_hanle_two_level_atom():
    """J = 0 -> 1 without stimulated emission: S_line w^(2) conj(rho^2_Q / rho^0_0)(J_u)
    equals the pinned two-level solution S^K_Q of (1 - eps) J^K_Q + eps B with the
    Hanle term, Gamma = 2 pi nu_L / A, for random anisotropic radiation and fields."""
    at = _atom2(0, 1)
    tab = mlpol.Tables(at, stimulated=False)
    rng = np.random.default_rng(4)
    n = 5
    kT = rng.uniform(0.4, 0.6, n)
    jr = rng.normal(size=(n, 1, 9)) * 0.3
    jr[..., 0] = rng.uniform(0.5, 1.5, size=(n, 1))
    jr[..., 1:4] = 0.0
    bv = rng.normal(size=(n, 3)) * 5
    x = tab.solve(tab.matrix(kT, jr, bv))
    xc = tab.to_complex(x)
    pops = tab.populations(x)
    Sw = pops[:, 1] / 3 / pops[:, 0]                 # source function without stimulated emission
    s2 = {Q: np.conj(xc[:, tab.idx[(1, 2, Q)]]) / xc[:, tab.idx[(1, 0, 0)]].real * Sw for Q in (0, 1, 2)}
    mine = np.stack([Sw, s2[0].real, s2[1].real, s2[1].imag, s2[2].real, s2[2].imag], -1)
    cul, _ = ml.collision_rates(at, kT)
    eps = cul[0] / (at["A"][0] + cul[0])
    shape = (2, 1, n)

    def rep(a):
        return np.broadcast_to(a, shape).copy()
    atm = dict(nx=n, ny=1, nz=2, lx=1.0, ly=1.0, z=np.array([0.0, 1.0]), chi=np.ones(shape), vel=np.zeros(shape),
               eps=rep(eps), bpl=rep(np.exp(-3.1 / kT)), bx=rep(bv[:, 0]), by=rep(bv[:, 1]), bz=rep(bv[:, 2]),
               zeta=0.0, gbar=1.0, bcrit=at["A"][0] / (2 * np.pi * mlpol.NU_L_PER_G))
    p = oracle.Problem(atm, 1, 1, 1, 3)
    jk6 = np.zeros(shape + (6,))
    jk6[..., 0] = rep(jr[:, 0, 0])
    for k, c in zip(range(1, 6), range(4, 9)):
        jk6[..., k] = rep(jr[:, 0, c])
    rho = np.zeros(shape + (6,))
    rho[..., 0] = 1.0
    S1, _ = oracle.see_update(p, jk6, np.zeros(shape), rho)
    assert np.allclose(mine, S1[0, 0], rtol=1e-10, atol=1e-12)


def test_dark_states_of_the_dipole_selection_rules():
    """A J = 1 lower level with only m = 0 populated absorbs no light travelling
    along z (only sigma components, m -> M = +-1 to J = 0 needs M = 0) and no pi
    light towards a J = 1 upper level ((1 1 1; 0 0 0) = 0); an upper J = 1 level
    with only M = 0 populated is not stimulated to a J = 0 level by light along
    z. The bright counterparts do absorb or emit."""
    # absorption J_l = 1 -> J_u = 0, beam along z (unpolarized)
    at = _atom2(1, 0)
    tab = mlpol.Tables(at)
    x = _sublevels(tab, 0, [0.0, 1.0, 0.0])
    z_beam = _beam(1.0, 0.0, [1.0, 0.0, 0.0])[None, None, :]
    Mc = tab.matrix(np.array([10.0]), z_beam, np.zeros((1, 3))) - tab.Ms - tab.collisions(np.array([10.0]))
    y = Mc[0] @ tab.to_complex(x)
    assert np.max(np.abs(y)) < 1e-9 * tab.Blu[0]
    xb = _sublevels(tab, 0, [1.0, 0.0, 0.0])        # m = -1 absorbs
    assert np.max(np.abs(Mc[0] @ tab.to_complex(xb))) > 0.1 * tab.Blu[0]
    # absorption J_l = 1 -> J_u = 1, pi light: beam along x polarized along z (Stokes Q = I for e_a = -z)
    at = _atom2(1, 1)
    tab = mlpol.Tables(at)
    x = _sublevels(tab, 0, [0.0, 1.0, 0.0])
    pi_beam = _beam(0.0, 0.0, [1.0, 1.0, 0.0])[None, None, :]
    Mc = tab.matrix(np.array([10.0]), pi_beam, np.zeros((1, 3))) - tab.Ms - tab.collisions(np.array([10.0]))
    assert np.max(np.abs(Mc[0] @ tab.to_complex(x))) < 1e-9 * tab.Blu[0]
    sigma_beam = _beam(0.0, 0.0, [1.0, -1.0, 0.0])[None, None, :]
    Mc2 = tab.matrix(np.array([10.0]), sigma_beam, np.zeros((1, 3))) - tab.Ms - tab.collisions(np.array([10.0]))
    assert np.max(np.abs(Mc2[0] @ tab.to_complex(x))) > 0.1 * tab.Blu[0]
    # stimulated emission J_u = 1 (M = 0 only) -> J_l = 0, beam along z
    at = _atom2(0, 1)
    tab = mlpol.Tables(at)
    x = _sublevels(tab, 1, [0.0, 1.0, 0.0])
    Mc = tab.matrix(np.array([10.0]), z_beam, np.zeros((1, 3))) - tab.Ms - tab.collisions(np.array([10.0]))
    assert np.max(np.abs(Mc[0] @ tab.to_complex(x))) < 1e-9 * tab.Bul[0]
    xb = _sublevels(tab, 1, [1.0, 0.0, 0.0])
    assert np.max(np.abs(Mc[0] @ tab.to_complex(xb))) > 0.1 * tab.Bul[0]


def test_lte_is_a_fixed_point_for_any_field():
    atom = synth.multilevel_atom(seed=5)
    tab = mlpol.Tables(atom)
    rng = np.random.default_rng(6)
    kT = rng.uniform(0.45, 0.55, 4)
    x = mlpol.lte_unknowns(tab, kT)
    jb = np.zeros((4, 4, 9))
    jb[..., 0] = ml.planck(atom, kT)
    new, change = mlpol.see_update(tab, kT, x, jb, rng.uniform(0, 0.9, (4, 4)), rng.normal(size=(4, 3)) * 30)
    assert change < 1e-12
    assert np.max(np.abs(new - x)) < 1e-12 * np.max(np.abs(x))


def test_iteration_reaches_a_solution_of_the_plain_rate_equations():
    atm = synth.multilevel_box(4, 4, 8, seed=2, tau_top=1e-2, tau_bot=1e2)
    atom = synth.multilevel_atom(seed=3, eps_range=(3e-2, 1e-1))
    tab = mlpol.Tables(atom)
    quad = (2, 4, 5)
    x = mlpol.lte_unknowns(tab, atm["kT"])
    for _ in range(200):
        x, change = mlpol.iterate(atm, atom, tab, x, quad, 1)
        if change < 1e-11:
            break
    assert change < 1e-11
    bvec = np.stack([atm["bx"], atm["by"], atm["bz"]], -1)
    jbar, _ = mlpol.formal_solve_lines(atm, atom, tab, x, quad)
    plain = tab.solve(tab.matrix(atm["kT"], jbar, bvec))
    assert np.max(np.abs(plain - x)) < 1e-8 * np.max(np.abs(x))
    # the anisotropic radiation polarizes the levels (alignment well above rounding)
    rb = mlpol.real_basis(atom)
    k20 = rb.index((3, 2, 0, 0))
    assert np.max(np.abs(x[..., k20] / x[..., rb.index((3, 0, 0, 0))])) > 1e-4


@pytest.mark.parametrize("Ju,Jl", [(1, 1), (1, 2), (2, 1), (2, 2), (1.5, 0.5)])
def test_spontaneous_emission_follows_the_sublevel_branching_ratios(Ju, Jl):
    """Spontaneous emission from an upper level with sublevel populations p_M
    (no coherences) fills lower sublevel m at the rate A sum_M (2Ju+1)
    (Ju Jl 1; -M m M-m)^2 p_M (Wigner-Eckart); the multipoles of that
    distribution are what the rate equations transfer."""
    at = _atom2(Jl, Ju)
    tab = mlpol.Tables(at)
    rng = np.random.default_rng(int(10 * Ju + Jl))
    p = rng.uniform(0.1, 1.0, int(round(2 * Ju + 1)))
    x = _sublevels(tab, 1, p)
    y = (tab.Ms @ tab.to_complex(x))                 # spontaneous terms only
    Mu = np.arange(-Ju, Ju + 1)
    ml_ = np.arange(-Jl, Jl + 1)
    gain = np.array([sum(at["A"][0] * (2 * Ju + 1) * w3j(Ju, Jl, 1, -M, m, M - m) ** 2 * pM for M, pM in zip(Mu, p))
                     for m in ml_])
    want = tab.to_complex(_sublevels(tab, 0, gain))
    lower = [k for k, (i, K, Q) in enumerate(tab.cb) if i == 0]
    assert np.allclose(y[lower], want[lower], rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))


def test_strong_collisions_depolarize_every_level():
    atom = synth.multilevel_atom(seed=7)
    atom["eps"] = np.full(4, 1.0 - 1e-9)
    tab = mlpol.Tables(atom)
    kT = np.array([0.5])
    jb = np.zeros((1, 4, 9))
    jb[..., 0] = ml.planck(atom, kT)
    jb[..., 4:9] = 0.3 * jb[..., :1]               # strongly anisotropic radiation
    x = tab.solve(tab.matrix(kT, jb, np.array([[3.0, -2.0, 5.0]])))
    rb = mlpol.real_basis(atom)
    pol = [k for k, (i, K, Q, part) in enumerate(rb) if K > 0]
    assert np.max(np.abs(x[0, pol])) < 1e-7 * np.max(np.abs(x))
    assert np.allclose(tab.populations(x), ml.lte_populations(atom, kT), rtol=1e-6)


def test_update_keeps_populations_positive_under_strong_anisotropy():
    """LTE start in optically thick layers (Lambda-bar* near 1) under strongly
    anisotropic radiation (|J^2_Q| / J^0_0 up to 0.3): the two-block update keeps
    every population positive (solving populations and multipoles in one system
    pairs the small J_eff with the full anisotropy and drives some negative)."""
    atom = synth.multilevel_atom(seed=0)
    tab = mlpol.Tables(atom)
    rng = np.random.default_rng(11)
    n = 400
    kT = rng.uniform(0.45, 0.55, n)
    x = mlpol.lte_unknowns(tab, kT)
    B = ml.planck(atom, kT)
    ls = 1.0 - 10 ** rng.uniform(-4, -1, (n, 4))
    jb = np.zeros((n, 4, 9))
    # J = Lambda* S + a positive remainder (J_eff >= 0, as a formal solution gives)
    jb[..., 0] = ls * B + (1 - ls) * B * rng.uniform(0.2, 1.0, (n, 4))
    jb[..., 4:9] = jb[..., :1] * rng.uniform(-0.3, 0.3, (n, 4, 5))
    bvec = rng.normal(size=(n, 3)) * 30
    new, _ = mlpol.see_update(tab, kT, x, jb, ls, bvec)
    assert np.min(tab.populations(new)) > 0
    # the single-system solve of the same equations goes negative for some of these voxels
    S_old = ml.source_function(atom, tab.populations(x))
    one = tab.solve(tab.matrix(kT, jb, bvec, ls, S_old))
    assert np.min(tab.populations(one)) < 0


def test_multigrid_cycles_reach_the_fixed_point_faster_than_jacobi():
    """Polarized five-level atom on 8x8x17 -> 4x4x9 -> 2x2x5: three V-cycles leave
    a residual f - A(x) well below Jacobi's at equal fine-grid cost; six more reach
    a solution of the plain rate equations that a further cycle leaves in place."""
    quad = (2, 4, 5)
    atm = synth.multilevel_box(8, 8, 17, seed=2, tau_top=1e-2, tau_bot=1e2)
    atm["zeta"] = 5e-5
    atom = synth.multilevel_atom(seed=3, eps_range=(1e-2, 3e-2))
    tab = mlpol.Tables(atom)
    x0 = mlpol.lte_unknowns(tab, atm["kT"])
    levels = ml.hierarchy(atm, 3)
    f = mlpol.f_fine(tab, x0.shape[:-1])

    def res(x):
        return np.max(np.abs(f - mlpol.apply_A(atm, atom, tab, x, quad)))
    x, y = x0.copy(), x0.copy()
    for _ in range(3):
        x = mlpol.vcycle(levels, atom, tab, quad, x)
        y, _ = mlpol.iterate(atm, atom, tab, y, quad, 7)
    assert res(x) * 30 < res(y)
    for _ in range(6):
        x = mlpol.vcycle(levels, atom, tab, quad, x)
    bvec = np.stack([atm["bx"], atm["by"], atm["bz"]], -1)
    jbar, _ = mlpol.formal_solve_lines(atm, atom, tab, x, quad)
    plain = tab.solve(tab.matrix(atm["kT"], jbar, bvec))
    assert np.max(np.abs(plain - x)) < 1e-8 * np.max(np.abs(x))
    x2 = mlpol.vcycle(levels, atom, tab, quad, x)
    assert np.max(np.abs(x2 - x)) < 1e-9 * np.max(np.abs(x))


def _eta_ratios(d5, mu, chi):
    """eta_i / eta_0 (i = I, Q, U) for dichroism multipoles d5 along (mu, chi)"""
    t = oracle.tkq(mu, chi)
    d6 = np.array([1.0, *d5])
    out = []
    for i in range(3):
        a = d6 if i == 0 else np.concatenate([[0.0], d6[1:]])
        out.append(t[i, 0] * a[0] + t[i, 1] * a[1] + 2 * (t[i, 2] * a[2] + t[i, 3] * a[3]) +
                   2 * (t[i, 4] * a[4] + t[i, 5] * a[5]))
    return np.array(out)


def test_dichroism_follows_the_selection_rules():
    """Absorption from a J = 1 lower level with only m = 0 populated towards J = 0
    (a pure pi transition): nothing is absorbed along z (eta_I = 0) and, along x,
    only light polarized along z (eta_I = eta_Q, reference direction e_a = -z). The
    same holds for stimulated emission from a J = 1 upper level with only M = 0
    populated towards J = 0. An unpolarized lower level gives no dichroism."""
    at = _atom2(1, 0)
    tab = mlpol.Tables(at)
    x = _sublevels(tab, 0, [0.0, 1.0, 0.0])
    d = mlpol.line_dichroism(tab, x, 0)
    assert abs(_eta_ratios(d, 1.0, 0.3)[0]) < 1e-12
    e = _eta_ratios(d, 0.0, 0.0)
    assert abs(e[0] - e[1]) < 1e-12 and e[0] > 0.5 and abs(e[2]) < 1e-12
    assert np.max(np.abs(mlpol.line_dichroism(tab, _sublevels(tab, 0, [1.0, 1.0, 1.0]), 0))) < 1e-14
    # stimulated emission (an inverted upper level alone: negative absorption, the same pattern)
    at = _atom2(0, 1)
    tab = mlpol.Tables(at)
    x = _sublevels(tab, 1, [0.0, 1.0, 0.0])
    d = mlpol.line_dichroism(tab, x, 0)
    assert abs(_eta_ratios(d, 1.0, 0.3)[0]) < 1e-12
    e = _eta_ratios(d, 0.0, 1.1)
    assert abs(e[0] - e[1]) < 1e-12 and e[0] > 0.5
