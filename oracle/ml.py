"""Multilevel atom without polarization: the non-LTE problem of the first kind
(populations only), which Sec. 1 names as the code's spectroscopy option and
as the particular case of the polarized multilevel problem with rho^0_0 alone.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline and reference legs, never by the product path.

The paper states this problem by reference (Sec. 2; its Eq. 2 with the
populations as the unknowns). The model written out here, one reading per
item:

* levels i with weights g_i = 2 J_i + 1 and energies E_i (eV); populations
  n_i per voxel with sum_i n_i = 1 (the conservation row);
* lines (u, l) with frequency proportional to dE = E_u - E_l; intensities in
  units of 2 h nu^3 / c^2 of the reference line (line 0), so that with
  r = dE / dE_ref the Planck function of a line is B = r^3 / (exp(dE/kT) - 1)
  and A_ul / B_ul = r^3;
* line-centre opacity chi_ul = chi s_ul (n_l - n_u g_l / g_u): chi is the
  atmosphere's opacity scale and s_ul = [(g_u / g_l) A_ul / dE^2] / [the
  same for the reference line] (h nu B_lu scales as (g_u / g_l) A_ul / nu^2);
* line source function S_ul = r^3 n_u / (n_l g_u / g_l - n_u) (complete
  redistribution, equal absorption and emission profiles);
* collisions on the line transitions: C_ul = eps A_ul / (1 - eps) with the
  line's eps = C / (A + C), and C_lu = (g_u / g_l) exp(-dE / kT) C_ul;
* boundaries as for the two-level atom: I = B_ul(T) entering at the bottom,
  nothing at the top.

Each line is one unpolarized formal solution (the two-level formal solver of
this package, with chi_ul, S_ul and B_ul). The Jacobi update is the
preconditioned (linear) form of the rate equations: with J_eff = Jbar -
Lambda-bar* S_old per line, the radiative rates P_ul = A_ul (1 - Lambda-bar*)
+ B_ul J_eff and P_lu = B_lu J_eff make the rate equations linear in the new
populations (the net radiative rate n_u A - (n_l B_lu - n_u B_ul) Jbar with
Jbar = J_eff + Lambda-bar* S and (n_l B_lu - n_u B_ul) S = n_u A); the
equation of level 0 is replaced by sum_i n_i = 1. For two levels this is the
two-level update of this package with eps' = C'/(A + C'), C' = C_ul (1 -
exp(-dE/kT)).

The non-linear multigrid cycle of Sec. 5 (Eqs. 30-34) carries over with the
populations as the unknowns: A(n) = f with A(n)_0 = sum_i n_i and A(n)_i =
(M n)_i (the plain rates of the formal solution's Jbar) for i >= 1, f = (1, 0,
..., 0) on the finest grid and f = A_c(R n) + R r on a coarser one, whose
Jacobi update takes f as the right-hand side; the coarse atmospheres (opacity
scale, temperature, velocity) are the fine values at the coincident nodes and
the grid transfer operators are those of oracle/mg.py.

Pins (tests/test_oracle_ml.py): strong collisions give Boltzmann
populations; LTE populations have S = B; Planckian radiation is a fixed point
of the update; rate-matrix columns sum to zero; the two-level case equals the
pinned two-level update; the emissivity depends on the upper population
alone; the converged populations satisfy the rate equations without
preconditioning; V-cycles reach that solution faster than Jacobi iterations
of equal cost and leave it unchanged.
"""
import numpy as np

from . import Problem, formal_solve


def line_tables(atom):
    """g (per level), dE, r = dE/dE_ref and the opacity strengths s (per line)."""
    J = np.asarray(atom["J"])
    g = 2.0 * J + 1.0
    E = np.asarray(atom["E"], dtype=np.float64)
    u, l = atom["lines"][:, 0], atom["lines"][:, 1]
    dE = E[u] - E[l]
    r = dE / dE[0]
    s = (g[u] / g[l]) * np.asarray(atom["A"]) / dE ** 2
    return g, dE, r, s / s[0]


def planck(atom, kT):
    """B_ul(T), shape kT.shape + (nline,)."""
    _, dE, r, _ = line_tables(atom)
    return r ** 3 / np.expm1(dE / np.asarray(kT)[..., None])


def lte_populations(atom, kT):
    """Boltzmann populations g_i exp(-E_i/kT), normalized to sum 1."""
    g, _, _, _ = line_tables(atom)
    E = np.asarray(atom["E"], dtype=np.float64)
    w = g * np.exp(-(E - E.min()) / np.asarray(kT)[..., None])
    return w / w.sum(-1, keepdims=True)


def line_opacity(atom, chi, pops):
    g, _, _, s = line_tables(atom)
    u, l = atom["lines"][:, 0], atom["lines"][:, 1]
    return np.asarray(chi)[..., None] * s * (pops[..., l] - pops[..., u] * g[l] / g[u])


def source_function(atom, pops):
    g, _, r, _ = line_tables(atom)
    u, l = atom["lines"][:, 0], atom["lines"][:, 1]
    return r ** 3 * pops[..., u] / (pops[..., l] * g[u] / g[l] - pops[..., u])


def collision_rates(atom, kT):
    """C_ul (nline,) and C_lu (kT.shape + (nline,))."""
    g, dE, _, _ = line_tables(atom)
    u, l = atom["lines"][:, 0], atom["lines"][:, 1]
    eps = np.asarray(atom["eps"])
    cul = eps / (1.0 - eps) * np.asarray(atom["A"])
    clu = (g[u] / g[l]) * np.exp(-dE / np.asarray(kT)[..., None]) * cul
    return cul, clu


def rate_matrix(atom, kT, jrad, lstar):
    """M with dn/dt = M n: the radiative rates P_ul = A (1 - lstar) + B_ul jrad,
    P_lu = B_lu jrad plus collisions (lstar = 0 and jrad = Jbar give the plain
    rate equations; lstar = Lambda-bar* and jrad = J_eff the preconditioned ones)."""
    g, _, r, _ = line_tables(atom)
    nlev = len(g)
    cul, clu = collision_rates(atom, kT)
    M = np.zeros(np.shape(kT) + (nlev, nlev))
    for k, (u, l) in enumerate(atom["lines"]):
        A = float(atom["A"][k])
        bul = A / r[k] ** 3
        blu = g[u] / g[l] * bul
        pul = A * (1.0 - lstar[..., k]) + bul * jrad[..., k] + cul[k]
        plu = blu * jrad[..., k] + clu[..., k]
        M[..., l, u] += pul
        M[..., u, u] -= pul
        M[..., u, l] += plu
        M[..., l, l] -= plu
    return M


def solve_populations(M):
    """n with M n = 0 and sum n = 1 (the row of level 0 replaced)."""
    M = M.copy()
    M[..., 0, :] = 1.0
    rhs = np.zeros(M.shape[:-1])
    rhs[..., 0] = 1.0
    return np.linalg.solve(M, rhs[..., None])[..., 0]


def see_update(atom, kT, pops, jbar, lstar, src=None):
    """One Jacobi update of the populations; returns (new, max relative change).
    src (per voxel, nlevel) replaces the right-hand side (1, 0, ..., 0) of the
    rate equations with their conservation row (the coarse-grid equations of
    the multigrid cycle)."""
    jeff = jbar - lstar * source_function(atom, pops)
    M = rate_matrix(atom, kT, jeff, lstar)
    if src is None:
        new = solve_populations(M)
    else:
        M = M.copy()
        M[..., 0, :] = 1.0
        new = np.linalg.solve(M, np.asarray(src)[..., None])[..., 0]
    return new, float(np.max(np.abs(new - pops) / np.abs(pops)))


def rate_operator(atom, kT, pops, jbar):
    """A(n) of the rate equations written as A(n) = (1, 0, ..., 0): row 0 is
    sum_i n_i, rows i >= 1 are (M n)_i with the plain radiative rates of Jbar."""
    M = rate_matrix(atom, kT, jbar, np.zeros_like(jbar))
    An = np.einsum("...ij,...j->...i", M, pops)
    An[..., 0] = pops.sum(-1)
    return An


def line_problem(atm, atom, pops, k, quad, sc_faces=0):
    """The two-level formal-solution problem of line k (opacity, Planck function);
    sc_faces: M and P on the first cell face crossed (Sec. 3.1), as for the two-level atom."""
    a = dict(atm)
    a["chi"] = line_opacity(atom, atm["chi"], pops)[..., k]
    a["bpl"] = planck(atom, atm["kT"])[..., k]
    a["eps"] = np.ones_like(a["chi"])
    return Problem(a, 0, *quad, sc_faces=sc_faces)


def formal_solve_lines(atm, atom, pops, quad, sc_faces=0):
    """Jbar and Lambda-bar* of every line, shape (nz, ny, nx, nline)."""
    S = source_function(atom, pops)
    nline = len(atom["lines"])
    jbar = np.zeros(pops.shape[:-1] + (nline,))
    lstar = np.zeros_like(jbar)
    for k in range(nline):
        p = line_problem(atm, atom, pops, k, quad, sc_faces)
        j, ls = formal_solve(p, S[..., k:k + 1])
        jbar[..., k] = j[..., 0]
        lstar[..., k] = ls
    return jbar, lstar


def iterate(atm, atom, pops, quad, n):
    """n Jacobi iterations from pops; returns (pops, last change)."""
    change = None
    for _ in range(n):
        jbar, lstar = formal_solve_lines(atm, atom, pops, quad)
        pops, change = see_update(atom, atm["kT"], pops, jbar, lstar)
    return pops, change


# ---------------------------------------------------------------- multigrid (Sec. 5)
# The non-linear multigrid cycle of Sec. 5 with the populations as the
# unknowns: A(n) = f with f = (1, 0, ..., 0) on the finest grid; the grid
# transfer operators are those of oracle/mg.py.

class MlLevel:
    def __init__(self, atm):
        self.atm = atm
        self.shape = (atm["nz"], atm["ny"], atm["nx"])


def coarsen(atm):
    """Coarse atmosphere: the fine values at the coincident nodes (coarse node
    (i, j, k) = fine node (2i, 2j, 2k))."""
    from .mg import coarse_nz
    nz, ny, nx = atm["nz"], atm["ny"], atm["nx"]
    assert nx % 2 == 0 and ny % 2 == 0
    ncz = coarse_nz(nz)
    c = dict(atm)
    c.update(nx=nx // 2, ny=ny // 2, nz=ncz, z=np.asarray(atm["z"])[0:2 * ncz:2])
    for k in ("chi", "kT", "vel", "bx", "by", "bz"):
        if atm.get(k) is not None:
            c[k] = np.ascontiguousarray(np.asarray(atm[k])[0:2 * ncz:2, 0::2, 0::2])
    return c


def hierarchy(atm, nlevels):
    levels = [MlLevel(atm)]
    for _ in range(nlevels - 1):
        levels.append(MlLevel(coarsen(levels[-1].atm)))
    return levels


def apply_A(atm, atom, pops, quad):
    jbar, _ = formal_solve_lines(atm, atom, pops, quad)
    return rate_operator(atom, atm["kT"], pops, jbar)


def f_fine(shape, nlevel):
    f = np.zeros(tuple(shape) + (nlevel,))
    f[..., 0] = 1.0
    return f


def jacobi(atm, atom, pops, quad, src, n):
    change = None
    for _ in range(n):
        jbar, lstar = formal_solve_lines(atm, atom, pops, quad)
        pops, change = see_update(atom, atm["kT"], pops, jbar, lstar, src)
    return pops, change


def vcycle(levels, atom, quad, pops, src=None, l=0, npre=2, npost=4, ncoarse=8, order=1):
    """One V-cycle from level l down to the coarsest (Eqs. 30-34); returns the
    new populations of level l. src None on the finest level: f = (1, 0, ...)."""
    from .mg import prolong, restrict
    lev = levels[l]
    f = f_fine(lev.shape, pops.shape[-1]) if src is None else src
    if l == len(levels) - 1:
        pops, _ = jacobi(lev.atm, atom, pops, quad, f, ncoarse)
        return pops
    pops, _ = jacobi(lev.atm, atom, pops, quad, f, npre)
    r = f - apply_A(lev.atm, atom, pops, quad)
    coarse = levels[l + 1]
    n_c0 = restrict(lev, pops)
    f_c = apply_A(coarse.atm, atom, n_c0, quad) + restrict(lev, r)
    n_c = vcycle(levels, atom, quad, n_c0, f_c, l + 1, npre, npost, ncoarse, order)
    pops = pops + prolong(lev, n_c - n_c0, order)
    pops, _ = jacobi(lev.atm, atom, pops, quad, f, npost)
    return pops
