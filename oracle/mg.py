"""Non-linear multigrid (FAS) V-cycle of the oracle (test infrastructure only).

Sec. 5 of Stepan & Trujillo Bueno (2013): with the statistical-equilibrium
equations written as A_l(rho) = f_l on grid level l (A from the formal
solution, f = eps B delta_K0 on the finest grid),
  residual         r_l = f_l - A_l(rho_l)                                  (Eq. 30)
  coarse equation  A_{l-1}(rho') = A_{l-1}(R rho_l) + R r_l                (Eq. 33)
  correction       rho_l <- rho_l + P (rho' - R rho_l)                     (Eq. 34)
with Jacobi smoothing before and after the coarse-grid correction (Sec. 5.3:
2 pre- and 4 post-smoothing iterations). The coarse grid keeps every other
node on each axis (coarse node (i, j, k) = fine node (2i, 2j, 2k), Sec. 5.1);
the atmosphere on a coarse grid is the fine one at those nodes.

Prolongation P (Sec. 5.2), one of the two operators the paper names:
tri-linear -- a fine node that coincides with a coarse node takes its value,
others interpolate linearly along each axis in which they fall between coarse
nodes (periodic in x and y; linear in the height z). With an even number of
fine planes the top fine plane lies above the coarse grid and takes the linear
extrapolation of the two top coarse planes. Tri-cubic-centered -- the same with
the cubic through the four nearest coarse nodes of each axis (in z the four
planes around the fine plane, the four innermost next to the bottom and top,
the top four for the extrapolated plane; at least four coarse nodes per axis).
Restriction R (both cases): the transpose of the tri-linear P normalized so
that a constant is restricted to itself (the adjoint of the tri-linear
prolongation over the 3^3 fine nodes around a coarse node; fewer at the bottom
and top).

Nested multigrid (Sec. 5.1, the nested method): the coarsest grid's own problem
is solved first (Jacobi), and each finer level in turn starts from the
prolongation of the coarser level's solution and runs V-cycles with itself as
the finest grid.

The operators are written as 1D matrices per axis (built node by node from the
definition above) applied along each axis; the V-cycle calls the oracle's
formal solution and statistical-equilibrium routines in the order above.
"""
import numpy as np

from . import Problem, formal_solve, nl_of, see_apply, see_update_src


def coarse_nz(nz):
    return (nz + 1) // 2 if nz % 2 else nz // 2


def prolong_1d_periodic(nf):
    """nf x nf/2 matrix: even fine node -> its coarse node; odd -> mean of the two neighbours."""
    assert nf % 2 == 0
    nc = nf // 2
    P = np.zeros((nf, nc))
    for i in range(nf):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, (i - 1) // 2] += 0.5
            P[i, ((i + 1) // 2) % nc] += 0.5
    return P


def prolong_1d_z(zf):
    """nz x nz_c matrix of linear interpolation in the height z between coarse planes."""
    nf = len(zf)
    nc = coarse_nz(nf)
    zc = zf[0:2 * nc:2]
    P = np.zeros((nf, nc))
    for k in range(nf):
        if k % 2 == 0:
            P[k, k // 2] = 1.0
            continue
        k0 = (k - 1) // 2
        if k0 + 1 >= nc:            # above the top coarse plane: extrapolate from the top two
            k0 = nc - 2
        k1 = k0 + 1
        t = (zf[k] - zc[k0]) / (zc[k1] - zc[k0])
        P[k, k0] = 1.0 - t
        P[k, k1] = t
    return P


def _lagrange(xs, x):
    """weights at x of the Lagrange polynomial through the nodes xs"""
    w = np.ones(len(xs))
    for a in range(len(xs)):
        for b in range(len(xs)):
            if a != b:
                w[a] *= (x - xs[b]) / (xs[a] - xs[b])
    return w


def prolong_1d_periodic_cubic(nf):
    """nf x nf/2 matrix: even fine node -> its coarse node; odd -> the cubic through
    the four nearest coarse nodes (unit spacing, periodic)."""
    assert nf % 2 == 0
    nc = nf // 2
    assert nc >= 4
    w = _lagrange(np.array([-1.0, 0.0, 1.0, 2.0]), 0.5)
    P = np.zeros((nf, nc))
    for i in range(nf):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            left = (i - 1) // 2
            for off in range(4):
                P[i, (left - 1 + off) % nc] += w[off]
    return P


def prolong_1d_z_cubic(zf):
    """nz x nz_c matrix of cubic interpolation in the height z through four coarse planes."""
    nf = len(zf)
    nc = coarse_nz(nf)
    assert nc >= 4
    zc = np.asarray(zf)[0:2 * nc:2]
    P = np.zeros((nf, nc))
    for k in range(nf):
        if k % 2 == 0:
            P[k, k // 2] = 1.0
            continue
        s = min(max((k - 1) // 2 - 1, 0), nc - 4)
        P[k, s:s + 4] = _lagrange(zc[s:s + 4], zf[k])
    return P


class Level:
    """One grid level: the problem, its atmosphere and the prolongation from the next coarser level."""

    def __init__(self, atm, model, quad):
        self.atm = atm
        self.model = model
        self.quad = quad
        self.prob = Problem(atm, model, *quad)
        self.shape = self.prob.shape


def coarsen(atm):
    """Coarse-grid atmosphere: every other node on each axis (injection)."""
    nz, ny, nx = atm["nz"], atm["ny"], atm["nx"]
    assert nx % 2 == 0 and ny % 2 == 0
    ncz = coarse_nz(nz)
    c = dict(atm)
    c.update(nx=nx // 2, ny=ny // 2, nz=ncz, z=np.asarray(atm["z"])[0:2 * ncz:2])
    for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz"):
        if atm.get(k) is not None:
            c[k] = np.ascontiguousarray(np.asarray(atm[k])[0:2 * ncz:2, 0::2, 0::2])
    return c


def hierarchy(atm, model, quad, nlevels):
    """Levels from the finest (index 0) to the coarsest."""
    levels = [Level(atm, model, quad)]
    for _ in range(nlevels - 1):
        levels.append(Level(coarsen(levels[-1].atm), model, quad))
    return levels


def _mats(fine, order=1):
    a = fine.atm
    if order == 3:
        return (prolong_1d_z_cubic(np.asarray(a["z"])), prolong_1d_periodic_cubic(a["ny"]),
                prolong_1d_periodic_cubic(a["nx"]))
    return (prolong_1d_z(np.asarray(a["z"])), prolong_1d_periodic(a["ny"]), prolong_1d_periodic(a["nx"]))


def prolong(fine, coarse_field, order=1):
    """P applied to a coarse field (nzc, nyc, nxc, nl) -> fine field; order 1
    tri-linear, 3 tri-cubic-centered."""
    Pz, Py, Px = _mats(fine, order)
    return np.einsum("kK,jJ,iI,KJIc->kjic", Pz, Py, Px, coarse_field)


def restrict(fine, fine_field):
    """R = normalized transpose of P: fine field -> coarse field."""
    Pz, Py, Px = _mats(fine)
    num = np.einsum("kK,jJ,iI,kjic->KJIc", Pz, Py, Px, fine_field)
    den = np.einsum("K,J,I->KJI", Pz.sum(0), Py.sum(0), Px.sum(0))
    return num / den[..., None]


def apply_A(level, rho):
    """A(rho) on a level: formal solution for J, then the SEE operator."""
    jkq, _ = formal_solve(level.prob, rho)
    return see_apply(level.prob, jkq, rho)


def f_fine(level):
    """Right-hand side of the two-level problem: eps B delta_K0."""
    nl = nl_of(level.model)
    f = np.zeros(level.shape + (nl,))
    f[..., 0] = np.asarray(level.atm["eps"]) * np.asarray(level.atm["bpl"])
    return f


def jacobi(level, rho, src, n):
    mc = None
    for _ in range(n):
        jkq, ls = formal_solve(level.prob, rho)
        rho, mc = see_update_src(level.prob, jkq, ls, rho, src)
    return rho, mc


def vcycle(levels, rho, src=None, l=0, npre=2, npost=4, ncoarse=8, order=1):
    """One V-cycle from level l down to the coarsest; returns the new rho on level l.
    src None means the level's own problem, f = eps B delta_K0; order: prolongation."""
    lev = levels[l]
    f = f_fine(lev) if src is None else src
    if l == len(levels) - 1:
        rho, _ = jacobi(lev, rho, f, ncoarse)
        return rho
    rho, _ = jacobi(lev, rho, f, npre)
    r = f - apply_A(lev, rho)
    coarse = levels[l + 1]
    rho_c0 = restrict(lev, rho)
    f_c = apply_A(coarse, rho_c0) + restrict(lev, r)
    rho_c = vcycle(levels, rho_c0, f_c, l + 1, npre, npost, ncoarse, order)
    rho = rho + prolong(lev, rho_c - rho_c0, order)
    rho, _ = jacobi(lev, rho, f, npost)
    return rho


def nested(levels, rho_coarsest, ncycles=1, npre=2, npost=4, ncoarse=8, order=3):
    """Nested multigrid: ncoarse Jacobi iterations of the coarsest grid's own problem
    from rho_coarsest, then for each finer level the prolongation of the coarser
    solution followed by ncycles V-cycles with that level as the finest; returns rho
    on the finest level."""
    rho, _ = jacobi(levels[-1], rho_coarsest, f_fine(levels[-1]), ncoarse)
    for l in range(len(levels) - 2, -1, -1):
        rho = prolong(levels[l], rho, order)
        for _ in range(ncycles):
            rho = vcycle(levels, rho, None, l, npre, npost, ncoarse, order)
    return rho
