"""Polarized multilevel atom: statistical equilibrium of the multipolar
components rho^K_Q(J) of every level (K = 0 .. 2J, Q = -K .. K; no
interference between different levels), Sec. 2 with the radiative rates of
the multilevel atom the paper takes from LL04 (Sect. 7.2) -- test
infrastructure only.

The rate equations, in the multipole representation (rho^K_{-Q} = (-1)^Q
conj(rho^K_Q)), with J^{Kr}_{Qr} of each line (Kr = 0, 1, 2; the radiation
field tensors of Eq. 1) and 3j, 6j and 9j symbols (oracle/wigner.py):

  d rho^K_Q(J)/dt = -i w_J sum_Q' H^K_{QQ'}(b) rho^K_Q'(J)                   (Hanle)
      + sum_{l, KlQl} TA(J K Q; l Kl Ql) rho^Kl_Ql(l)                        (absorption from lower levels)
      + sum_{u, KuQu} [TE + TS](J K Q; u Ku Qu) rho^Ku_Qu(u)                 (emission from upper levels)
      - sum_{K'Q'} [RA + RE + RS](J K Q; K' Q') rho^K'_Q'(J)                 (relaxation)
      + collisions

  TA = (2Jl+1) B_lu sum_{KrQr} sqrt(3(2K+1)(2Kl+1)(2Kr+1)) (-1)^(Kl+Ql)
          {J Jl 1; J Jl 1; K Kl Kr} (K Kl Kr; -Q Ql -Qr) J^Kr_Qr
  TE = delta_{K Ku} delta_{Q Qu} (2Ju+1) A_ul (-1)^(1+Ju+J+K) {Ju Ju K; J J 1}
  TS = (2Ju+1) B_ul sum_{KrQr} sqrt(3(2K+1)(2Ku+1)(2Kr+1)) (-1)^(Kr+Ku+Qu)
          {Ju J 1; Ju J 1; Ku K Kr} (K Ku Kr; -Q Qu -Qr) J^Kr_Qr
  RA = (2J+1) sum_u B_lu sum_{KrQr} sqrt(3(2K+1)(2K'+1)(2Kr+1)) (-1)^(1+Ju-J+Kr+Q')
          {K K' Kr; J J J} {1 1 Kr; J J Ju} (K K' Kr; Q -Q' Qr) J^Kr_Qr
  RE = delta_{KK'} delta_{QQ'} sum_l A_ul
  RS = (2J+1) sum_l B_ul sum_{KrQr} sqrt(3(2K+1)(2K'+1)(2Kr+1)) (-1)^(1+Jl-J+Q')
          {K K' Kr; J J J} {1 1 Kr; J J Jl} (K K' Kr; Q -Q' Qr) J^Kr_Qr
  (RA and RS only for even K + K' + Kr.)

H^K is the matrix of the field direction b . J on rank-K multipoles (H_QQ =
Q b_z, H_{Q,Q-1} = (1/2)(b_x - i b_y) sqrt((K+Q)(K-Q+1)), H_{Q,Q+1} = (1/2)(b_x +
i b_y) sqrt((K-Q)(K+Q+1))) and w_J = 2 pi nu_L g_J the Larmor frequency of
the level (nu_L = 1.3996e6 Hz per gauss): for b along z, rho^K_Q turns as
e^{-i Q w_J t}, the counterclockwise precession of the atom about the field for
g_J > 0 (rho^K_Q transform as e^{-i Q alpha} under a rotation by alpha about z).
The two-level model of this package, to which the J = 0 -> 1 atom reduces,
has the same sense.
Collisions (a reading): inelastic collisions on the line transitions move
populations only (K = 0) and relax every multipole of the level they leave;
no elastic depolarization. Units as in oracle/ml.py (A in s^-1, intensities
in units of 2 h nu^3 / c^2 of line 0, B_ul = A_ul / r^3, B_lu = (g_u/g_l) B_ul).

Jacobi update (a reading; the paper's Jacobian method is that of its
multilevel 1D code): in two blocks. (1) The population equations (the K = 0
rows, the row of level 0 replaced by the trace sum_J sqrt(2J+1) rho^0_0(J) =
1) with Lambda-bar* preconditioning of the population (K = 0, Kr = 0) terms
exactly as the unpolarized multilevel update (J^0_0 -> J_eff = Jbar^0_0 -
Lambda-bar* S_old and A -> A (1 - Lambda-bar*) in the spontaneous K = 0 -> 0
transfer and relaxation), the K > 0 multipoles at their previous values;
(2) the K > 0 equations with the plain rates of Jbar and the new populations.
Solving both blocks at once would pair the small J_eff of optically thick
layers with the full anisotropy J^2_Q and can give negative populations.
Without polarization this is the update of oracle/ml.py; the fixed point is
that of the rate equations.

Line transfer (a reading): the emissivity of a line carries the upper level's
multipoles K = 0, 1, 2 (the two-level formal solver of this package, eps_i =
eta_I sum_KQ (-1)^Q T^K_Q S^K_-Q with S^K_Q = S_line w^(K) conj(rho^K_Q /
rho^0_0)(J_u), w^(K) = (-1)^(1+Jl+Ju) sqrt(3(2Ju+1)) {1 1 K; Ju Ju Jl}; the
orientation K = 1 enters Stokes V only, through T^1_Q(V, Omega) = sqrt(3/2)
Omega_Q); the absorption matrix carries the line's dichroism from the
alignment (K = 2) and orientation (K = 1) of its lower level (absorption, with
the factor (-1)^K of absorption against emission) and upper level (stimulated
emission), line_dichroism; the weak-field Zeeman term uses the field scaled by
the line's effective Lande factor (1 for every level here). The formal solution
gives J^Kr_Qr for Kr = 0, 1, 2 (J^1_Q from Stokes V).
"""
import numpy as np

from . import Problem, formal_solve
from . import ml
from .wigner import w3j, w6j, w9j

NU_L_PER_G = 1.3996e6          # Larmor frequency per gauss (Hz)


def _levels(atom):
    return [float(j) for j in atom["J"]]


def basis(atom):
    """complex unknowns: (level, K, Q) for every K <= 2J and Q = -K..K"""
    out = []
    for i, J in enumerate(_levels(atom)):
        for K in range(int(round(2 * J)) + 1):
            for Q in range(-K, K + 1):
                out.append((i, K, Q))
    return out


def real_basis(atom):
    """real unknowns: (level, K, Q, part) with Q >= 0 (part 0: real, 1: imaginary; Q = 0 real only)"""
    out = []
    for i, J in enumerate(_levels(atom)):
        for K in range(int(round(2 * J)) + 1):
            out.append((i, K, 0, 0))
            for Q in range(1, K + 1):
                out.append((i, K, Q, 0))
                out.append((i, K, Q, 1))
    return out


def _maps(atom):
    """C (complex from real, x = C r) and the row selection of the real equations"""
    cb = basis(atom)
    rb = real_basis(atom)
    cidx = {b: n for n, b in enumerate(cb)}
    C = np.zeros((len(cb), len(rb)), dtype=complex)
    for n, (i, K, Q, part) in enumerate(rb):
        if Q == 0:
            C[cidx[(i, K, 0)], n] = 1.0
            continue
        z = 1.0 if part == 0 else 1j
        C[cidx[(i, K, Q)], n] += z
        C[cidx[(i, K, -Q)], n] += (-1) ** Q * np.conj(z)
    rows = [(cidx[(i, K, Q)], part) for (i, K, Q, part) in rb]
    return C, rows


def jkq_index():
    """the radiation tensors (Kr, Qr) of a line, Kr = 0, 1, 2"""
    return [(Kr, Qr) for Kr in range(3) for Qr in range(-Kr, Kr + 1)]


def jkq_complex(jr):
    """real layout (J00, J10, Re J11, Im J11, J20, Re J21, Im J21, Re J22, Im J22) ->
    complex J^Kr_Qr for all Qr (J^K_-Q = (-1)^Q conj J^K_Q)"""
    jr = np.asarray(jr)
    out = {}
    out[(0, 0)] = jr[..., 0] + 0j
    out[(1, 0)] = jr[..., 1] + 0j
    out[(1, 1)] = jr[..., 2] + 1j * jr[..., 3]
    out[(2, 0)] = jr[..., 4] + 0j
    out[(2, 1)] = jr[..., 5] + 1j * jr[..., 6]
    out[(2, 2)] = jr[..., 7] + 1j * jr[..., 8]
    for K, Q in list(out):
        if Q > 0:
            out[(K, -Q)] = (-1) ** Q * np.conj(out[(K, Q)])
    return out


class Tables:
    """The rate equations as sums of fixed complex matrices: spontaneous and
    the per-line, per-(Kr, Qr) radiative matrices (split into the population
    part the preconditioning acts on and the rest), the Hanle matrices per
    field component, and the collisional matrices."""

    def __init__(self, atom, stimulated=True):
        self.atom = atom
        J = _levels(atom)
        self.J = J
        self.g = np.array([2 * j + 1 for j in J])
        cb = basis(atom)
        self.cb = cb
        n = len(cb)
        self.n = n
        idx = {b: k for k, b in enumerate(cb)}
        self.idx = idx
        g, dE, r, s = ml.line_tables(atom)
        lines = [(int(u), int(l)) for u, l in atom["lines"]]
        self.lines = lines
        nl = len(lines)
        jk = jkq_index()
        self.jk = jk
        A = np.asarray(atom["A"], dtype=np.float64)
        Bul = A / r ** 3
        Blu = np.array([g[u] / g[l] for u, l in lines]) * Bul
        # radiative matrices per line and (Kr, Qr); pop[...] holds the K = Kl = Kr = 0 parts
        self.Mr = np.zeros((nl, len(jk), n, n), dtype=complex)
        self.Mpop = np.zeros((nl, n, n), dtype=complex)       # coefficient of J^0_0 in population terms
        self.Ms = np.zeros((n, n), dtype=complex)             # spontaneous (all)
        self.Mspop = np.zeros((nl, n, n), dtype=complex)      # spontaneous K = 0 -> 0 parts per line
        for li, (u, l) in enumerate(lines):
            Ju, Jl = J[u], J[l]
            for a, (lev, K, Q) in enumerate(cb):
                if lev == u:
                    # absorption from the lower level into the upper level
                    for Kl in range(int(round(2 * Jl)) + 1):
                        for Ql in range(-Kl, Kl + 1):
                            b = idx[(l, Kl, Ql)]
                            for c, (Kr, Qr) in enumerate(jk):
                                v = ((2 * Jl + 1) * Blu[li] * np.sqrt(3 * (2 * K + 1) * (2 * Kl + 1) * (2 * Kr + 1)) *
                                     (-1) ** (Kl + Ql) * w9j(Ju, Jl, 1, Ju, Jl, 1, K, Kl, Kr) *
                                     w3j(K, Kl, Kr, -Q, Ql, -Qr))
                                if v != 0.0:
                                    self.Mr[li, c, a, b] += v
                                    if K == 0 and Kl == 0 and Kr == 0:
                                        self.Mpop[li, a, b] += v
                    # relaxation of the upper level: spontaneous and stimulated emission
                    self.Ms[a, a] -= A[li]
                    if K == 0:
                        self.Mspop[li, a, a] -= A[li]
                    if stimulated:
                        for Kp in range(int(round(2 * Ju)) + 1):
                            for Qp in range(-Kp, Kp + 1):
                                b = idx[(u, Kp, Qp)]
                                for c, (Kr, Qr) in enumerate(jk):
                                    if (K + Kp + Kr) % 2:
                                        continue
                                    v = ((2 * Ju + 1) * Bul[li] * np.sqrt(3 * (2 * K + 1) * (2 * Kp + 1) * (2 * Kr + 1)) *
                                         (-1) ** (1 + Jl - Ju + Qp) * w6j(K, Kp, Kr, Ju, Ju, Ju) *
                                         w6j(1, 1, Kr, Ju, Ju, Jl) * w3j(K, Kp, Kr, Q, -Qp, Qr))
                                    if v != 0.0:
                                        self.Mr[li, c, a, b] -= v
                                        if K == 0 and Kp == 0 and Kr == 0:
                                            self.Mpop[li, a, b] -= v
                if lev == l:
                    # spontaneous and stimulated emission from the upper level into the lower level
                    b = idx.get((u, K, Q))
                    if b is not None:
                        v = (2 * Ju + 1) * A[li] * (-1) ** (1 + Ju + Jl + K) * w6j(Ju, Ju, K, Jl, Jl, 1)
                        self.Ms[a, b] += v
                        if K == 0:
                            self.Mspop[li, a, b] += v
                    if stimulated:
                        for Ku in range(int(round(2 * Ju)) + 1):
                            for Qu in range(-Ku, Ku + 1):
                                b = idx[(u, Ku, Qu)]
                                for c, (Kr, Qr) in enumerate(jk):
                                    v = ((2 * Ju + 1) * Bul[li] * np.sqrt(3 * (2 * K + 1) * (2 * Ku + 1) * (2 * Kr + 1)) *
                                         (-1) ** (Kr + Ku + Qu) * w9j(Ju, Jl, 1, Ju, Jl, 1, Ku, K, Kr) *
                                         w3j(K, Ku, Kr, -Q, Qu, -Qr))
                                    if v != 0.0:
                                        self.Mr[li, c, a, b] += v
                                        if K == 0 and Ku == 0 and Kr == 0:
                                            self.Mpop[li, a, b] += v
                    # relaxation of the lower level by absorption
                    for Kp in range(int(round(2 * Jl)) + 1):
                        for Qp in range(-Kp, Kp + 1):
                            b = idx[(l, Kp, Qp)]
                            for c, (Kr, Qr) in enumerate(jk):
                                if (K + Kp + Kr) % 2:
                                    continue
                                v = ((2 * Jl + 1) * Blu[li] * np.sqrt(3 * (2 * K + 1) * (2 * Kp + 1) * (2 * Kr + 1)) *
                                     (-1) ** (1 + Ju - Jl + Kr + Qp) * w6j(K, Kp, Kr, Jl, Jl, Jl) *
                                     w6j(1, 1, Kr, Jl, Jl, Ju) * w3j(K, Kp, Kr, Q, -Qp, Qr))
                                if v != 0.0:
                                    self.Mr[li, c, a, b] -= v
                                    if K == 0 and Kp == 0 and Kr == 0:
                                        self.Mpop[li, a, b] -= v
        # Hanle: -i w_J H^K(b) per field component (b_x, b_y, b_z in gauss)
        self.Mh = np.zeros((3, n, n), dtype=complex)
        for a, (lev, K, Q) in enumerate(cb):
            wj = -2 * np.pi * NU_L_PER_G * 1.0         # -w_J, Lande factor 1 for every level
            for Qp in (Q - 1, Q, Q + 1):
                if abs(Qp) > K:
                    continue
                b = idx[(lev, K, Qp)]
                if Qp == Q:
                    self.Mh[2, a, b] += 1j * wj * Q
                elif Qp == Q - 1:
                    f = 0.5 * np.sqrt((K + Q) * (K - Q + 1))
                    self.Mh[0, a, b] += 1j * wj * f
                    self.Mh[1, a, b] += 1j * wj * f * (-1j)
                else:
                    f = 0.5 * np.sqrt((K - Q) * (K + Q + 1))
                    self.Mh[0, a, b] += 1j * wj * f
                    self.Mh[1, a, b] += 1j * wj * f * (1j)
        self.Bul, self.Blu, self.A, self.r3 = Bul, Blu, A, r ** 3
        self.C, self.rows = _maps(atom)
        self.trace = np.zeros(len(self.rows))
        rb = real_basis(atom)
        for k, (i, K, Q, part) in enumerate(rb):
            if K == 0:
                self.trace[k] = np.sqrt(self.g[i])
        self.row0 = rb.index((0, 0, 0, 0))

    def _collision_units(self):
        """the collisional matrix as C_ul terms (constant) plus unit C_lu terms per line"""
        cul, _ = ml.collision_rates(self.atom, np.array(1.0))
        n = self.n
        const = np.zeros((n, n), dtype=complex)
        unit = np.zeros((len(self.lines), n, n), dtype=complex)
        for li, (u, l) in enumerate(self.lines):
            gu, gl = self.g[u], self.g[l]
            a0u, a0l = self.idx[(u, 0, 0)], self.idx[(l, 0, 0)]
            # populations n = sqrt(2J+1) rho^0_0: dn_u = C_lu n_l - C_ul n_u; every
            # multipole of the level left relaxes
            unit[li, a0u, a0l] += np.sqrt(gl / gu)
            const[a0l, a0u] += cul[li] * np.sqrt(gu / gl)
            for a, (lev, K, Q) in enumerate(self.cb):
                if lev == u:
                    const[a, a] -= cul[li]
                elif lev == l:
                    unit[li, a, a] -= 1.0
        return const, unit

    def collisions(self, kT):
        """collisional matrix per voxel (kT.shape + (n, n)), complex"""
        const, unit = self._collision_units()
        _, clu = ml.collision_rates(self.atom, kT)
        return const + np.einsum("...l,lij->...ij", clu + 0j, unit)

    def matrix(self, kT, jbar, bvec, lstar=None, S_old=None):
        """complex rate matrix per voxel; jbar [..., nline, 9] real layout, bvec [..., 3];
        with lstar and S_old, the preconditioned population terms. The sum of
        source x matrix is one product over all sources."""
        nl, n = len(self.lines), self.n
        const, unit = self._collision_units()
        _, clu = ml.collision_rates(self.atom, kT)
        coefs, mats = [clu + 0j], [unit]
        jc = [jkq_complex(jbar[..., li, :]) for li in range(nl)]
        coefs.append(np.stack([jc[li][kq] for li in range(nl) for kq in self.jk], -1))
        mats.append(self.Mr.reshape(nl * len(self.jk), n, n))
        if lstar is not None:
            # J^0_0 -> J_eff and A -> A (1 - Lambda*) in the population terms
            coefs.append(-lstar * S_old + 0j)
            mats.append(self.Mpop)
            coefs.append(-lstar + 0j)
            mats.append(self.Mspop)
        coefs.append(np.asarray(bvec) + 0j)
        mats.append(self.Mh)
        cf = np.concatenate(coefs, -1)
        mt = np.concatenate(mats, 0)
        shape = cf.shape[:-1]
        M = (cf.reshape(-1, cf.shape[-1]) @ mt.reshape(mt.shape[0], n * n)).reshape(shape + (n, n))
        return M + const + self.Ms

    def real_system(self, Mc):
        """real matrix of the equations (rows: Q = 0 real parts; Q > 0 real and imaginary parts)"""
        Y = Mc @ self.C
        R = np.zeros(Y.shape[:-2] + (len(self.rows), Y.shape[-1]))
        for k, (ci, part) in enumerate(self.rows):
            R[..., k, :] = Y[..., ci, :].real if part == 0 else Y[..., ci, :].imag
        return R

    def solve(self, Mc, rhs=None):
        """real unknowns with the trace row replacing level 0's population equation"""
        R = self.real_system(Mc)
        R[..., self.row0, :] = self.trace
        b = np.zeros(R.shape[:-1])
        b[..., self.row0] = 1.0
        if rhs is not None:
            b = np.asarray(rhs)
        return np.linalg.solve(R, b[..., None])[..., 0]

    def populations(self, x):
        """n_i = sqrt(2J+1) rho^0_0 from real unknowns"""
        rb = real_basis(self.atom)
        return np.stack([np.sqrt(self.g[i]) * x[..., rb.index((i, 0, 0, 0))] for i in range(len(self.g))], -1)

    def to_complex(self, x):
        return x @ self.C.T


def line_source_multipoles(tab, x):
    """per line, the two-level formal solver's S^K_Q (real layout S00, S20, Re S21,
    Im S21, Re S22, Im S22): S_line w^(K) conj(rho^K_Q / rho^0_0)(J_u)"""
    atom = tab.atom
    pops = tab.populations(x)
    S = ml.source_function(atom, pops)
    xc = tab.to_complex(x)
    out = np.zeros(x.shape[:-1] + (len(tab.lines), 6))
    for li, (u, l) in enumerate(tab.lines):
        Ju, Jl = tab.J[u], tab.J[l]
        r00 = xc[..., tab.idx[(u, 0, 0)]].real
        out[..., li, 0] = S[..., li]
        if Ju < 1:
            continue
        w2 = (-1) ** int(round(1 + Jl + Ju)) * np.sqrt(3 * (2 * Ju + 1)) * w6j(1, 1, 2, Ju, Ju, Jl)
        s = {Q: np.conj(xc[..., tab.idx[(u, 2, Q)]]) / r00 * w2 * S[..., li] for Q in (0, 1, 2)}
        out[..., li, 1] = s[0].real
        out[..., li, 2], out[..., li, 3] = s[1].real, s[1].imag
        out[..., li, 4], out[..., li, 5] = s[2].real, s[2].imag
    return out


def _w(K, J, Jp):
    """w^(K)_{J J'} = (-1)^(1+J+J') sqrt(3(2J+1)) {1 1 K; J J J'} (0 where 2J < K)"""
    if 2 * J < K:
        return 0.0
    return (-1) ** int(round(1 + J + Jp)) * np.sqrt(3 * (2 * J + 1)) * w6j(1, 1, K, J, J, Jp)


def line_orientation_multipoles(tab, x):
    """per line, the orientation emission multipoles S^1_Q = S_line w^(1) conj(rho^1_Q /
    rho^0_0)(J_u) in the layout (S10, Re S11, Im S11)"""
    atom = tab.atom
    S = ml.source_function(atom, tab.populations(x))
    xc = tab.to_complex(x)
    out = np.zeros(x.shape[:-1] + (len(tab.lines), 3))
    for li, (u, l) in enumerate(tab.lines):
        Ju, Jl = tab.J[u], tab.J[l]
        if 2 * Ju < 1:
            continue
        r00 = xc[..., tab.idx[(u, 0, 0)]].real
        s = {Q: np.conj(xc[..., tab.idx[(u, 1, Q)]]) / r00 * _w(1, Ju, Jl) * S[..., li] for Q in (0, 1)}
        out[..., li, 0] = s[0].real
        out[..., li, 1], out[..., li, 2] = s[1].real, s[1].imag
    return out


def line_dichroism_orientation(tab, x, li):
    """the orientation dichroism multipoles of line li, D^1_Q in the layout (D10, Re D11,
    Im D11): eta_V gains eta_I sum_Q (-1)^Q T^1_Q(V, Omega) D^1_-Q with
      D^1_Q = conj([-B_lu sqrt(2Jl+1) w1(Jl, Ju) rho^1_Q(Jl) - B_ul sqrt(2Ju+1) w1(Ju, Jl) rho^1_Q(Ju)]
                    / [B_lu sqrt(2Jl+1) rho^0_0(Jl) - B_ul sqrt(2Ju+1) rho^0_0(Ju)])
    (line_dichroism with K = 1: the absorption term carries (-1)^K = -1)."""
    u, l = tab.lines[li]
    Ju, Jl = tab.J[u], tab.J[l]
    xc = tab.to_complex(x)
    al = tab.Blu[li] * np.sqrt(2 * Jl + 1)
    au = tab.Bul[li] * np.sqrt(2 * Ju + 1)
    den = al * xc[..., tab.idx[(l, 0, 0)]].real - au * xc[..., tab.idx[(u, 0, 0)]].real
    out = np.zeros(x.shape[:-1] + (3,))
    for Q, (kr, ki) in ((0, (0, None)), (1, (1, 2))):
        num = np.zeros(x.shape[:-1], dtype=complex)
        if 2 * Jl >= 1:
            num = num - al * _w(1, Jl, Ju) * xc[..., tab.idx[(l, 1, Q)]]
        if 2 * Ju >= 1:
            num = num - au * _w(1, Ju, Jl) * xc[..., tab.idx[(u, 1, Q)]]
        d = np.conj(num / den)
        out[..., kr] = np.real(d)
        if ki is not None:
            out[..., ki] = np.imag(d)
    return out


def line_dichroism(tab, x, li):
    """dichroism multipoles of line li in the formal solver's layout (D20, Re D21,
    Im D21, Re D22, Im D22): the alignment terms of the line's absorption (lower
    level) minus stimulated emission (upper level) relative to their K = 0 terms,
    eta_i = eta_I [delta_i0 + sum_Q (-1)^Q T^2_Q(i, Omega) D^2_-Q] with
      D^2_Q = conj([B_lu sqrt(2Jl+1) w2(Jl, Ju) rho^2_Q(Jl) - B_ul sqrt(2Ju+1) w2(Ju, Jl) rho^2_Q(Ju)]
                    / [B_lu sqrt(2Jl+1) rho^0_0(Jl) - B_ul sqrt(2Ju+1) rho^0_0(Ju)]),
    w2(J, J') = (-1)^(1+J+J') sqrt(3(2J+1)) {1 1 2; J J J'} (LL04's absorption and
    stimulated-emission coefficients, the (-1)^K of absorption being 1 for K = 2)."""
    u, l = tab.lines[li]
    Ju, Jl = tab.J[u], tab.J[l]
    xc = tab.to_complex(x)

    def w2(J, Jp):
        if J < 1:
            return 0.0
        return (-1) ** int(round(1 + J + Jp)) * np.sqrt(3 * (2 * J + 1)) * w6j(1, 1, 2, J, J, Jp)
    al = tab.Blu[li] * np.sqrt(2 * Jl + 1)
    au = tab.Bul[li] * np.sqrt(2 * Ju + 1)
    den = al * xc[..., tab.idx[(l, 0, 0)]].real - au * xc[..., tab.idx[(u, 0, 0)]].real
    out = np.zeros(x.shape[:-1] + (5,))
    for Q, (kr, ki) in ((0, (0, None)), (1, (1, 2)), (2, (3, 4))):
        num = np.zeros(x.shape[:-1], dtype=complex)
        if Jl >= 1:
            num = num + al * w2(Jl, Ju) * xc[..., tab.idx[(l, 2, Q)]]
        if Ju >= 1:
            num = num - au * w2(Ju, Jl) * xc[..., tab.idx[(u, 2, Q)]]
        d = np.conj(num / den)
        out[..., kr] = np.real(d)
        if ki is not None:
            out[..., ki] = np.imag(d)
    return out


def line_problem(atm, atom, tab, x, li, quad, dichroism=True, sc_faces=0):
    """the two-level polarized formal-solution problem of line li (with the line's
    dichroism from the atomic polarization of its levels unless dichroism=False);
    sc_faces: M and P on the first cell face crossed (Sec. 3.1)"""
    pops = tab.populations(x)
    a = dict(atm)
    a["chi"] = ml.line_opacity(atom, atm["chi"], pops)[..., li]
    a["bpl"] = ml.planck(atom, atm["kT"])[..., li]
    a["eps"] = np.ones_like(a["chi"])
    if dichroism:
        a["dich"] = line_dichroism(tab, x, li)
        a["dich1"] = line_dichroism_orientation(tab, x, li)
    a["orient"] = line_orientation_multipoles(tab, x)[..., li, :]
    return Problem(a, 1, *quad, sc_faces=sc_faces)


def formal_solve_lines(atm, atom, tab, x, quad, dichroism=True, sc_faces=0):
    """Jbar (real layout of jkq_complex, Kr = 0, 1, 2) and Lambda-bar* per line"""
    src = line_source_multipoles(tab, x)
    nline = len(tab.lines)
    shape = x.shape[:-1]
    jbar = np.zeros(shape + (nline, 9))
    lstar = np.zeros(shape + (nline,))
    for li in range(nline):
        p = line_problem(atm, atom, tab, x, li, quad, dichroism, sc_faces)
        j, ls, j1 = formal_solve(p, src[..., li, :], with_j1=True)
        # two-level layout (J00, J20, ReJ21, ImJ21, ReJ22, ImJ22) and J^1 -> Kr = 0, 1, 2 layout
        jbar[..., li, 0] = j[..., 0]
        jbar[..., li, 1:4] = j1
        jbar[..., li, 4:9] = j[..., 1:6]
        lstar[..., li] = ls
    return jbar, lstar


def see_update(tab, kT, x, jbar, lstar, bvec, src=None):
    """one Jacobi update in two blocks; returns (new real unknowns, max relative
    change of the populations). (1) the population equations (K = 0 rows,
    preconditioned, the trace row for level 0) with the K > 0 multipoles at their
    old values; (2) the K > 0 equations (plain rates) with the new populations.
    src (per voxel, nunk) replaces the right-hand side e_row0 (coarse-grid
    equations of the multigrid cycle)."""
    S_old = ml.source_function(tab.atom, tab.populations(x))
    R = tab.real_system(tab.matrix(kT, jbar, bvec, lstar, S_old))
    R[..., tab.row0, :] = tab.trace
    if src is None:
        b = np.zeros(R.shape[:-1])
        b[..., tab.row0] = 1.0
    else:
        b = np.array(src, dtype=np.float64)
    rb = real_basis(tab.atom)
    k0 = [k for k, (i, K, Q, part) in enumerate(rb) if K == 0]
    kp = [k for k, (i, K, Q, part) in enumerate(rb) if K > 0]
    r1 = b[..., k0] - np.einsum("...ij,...j->...i", R[..., k0, :][..., :, kp], x[..., kp])
    y = np.linalg.solve(R[..., k0, :][..., :, k0], r1[..., None])[..., 0]
    r2 = b[..., kp] - np.einsum("...ij,...j->...i", R[..., kp, :][..., :, k0], y)
    z = np.linalg.solve(R[..., kp, :][..., :, kp], r2[..., None])[..., 0]
    new = np.zeros_like(x)
    new[..., k0] = y
    new[..., kp] = z
    p0, p1 = tab.populations(x), tab.populations(new)
    return new, float(np.max(np.abs(p1 - p0) / np.abs(p0)))


def lte_unknowns(tab, kT):
    """Boltzmann populations, no atomic polarization"""
    pops = ml.lte_populations(tab.atom, kT)
    x = np.zeros(np.shape(kT) + (len(tab.rows),))
    rb = real_basis(tab.atom)
    for i in range(len(tab.g)):
        x[..., rb.index((i, 0, 0, 0))] = pops[..., i] / np.sqrt(tab.g[i])
    return x


def iterate(atm, atom, tab, x, quad, n):
    bvec = np.stack([atm["bx"], atm["by"], atm["bz"]], -1)
    change = None
    for _ in range(n):
        jbar, lstar = formal_solve_lines(atm, atom, tab, x, quad)
        x, change = see_update(tab, atm["kT"], x, jbar, lstar, bvec)
    return x, change


# ---------------------------------------------------------------- multigrid (Sec. 5)
# The cycle of oracle/ml.py with the real multipoles as the unknowns: A(x)_row0 =
# sum_J sqrt(2J+1) rho^0_0(J), the other rows the plain rate equations of the
# formal solution's Jbar; f = e_row0 on the finest grid.

def rate_operator(tab, kT, x, jbar, bvec):
    R = tab.real_system(tab.matrix(kT, jbar, bvec))
    R[..., tab.row0, :] = tab.trace
    return np.einsum("...ij,...j->...i", R, x)


def apply_A(atm, atom, tab, x, quad):
    jbar, _ = formal_solve_lines(atm, atom, tab, x, quad)
    return rate_operator(tab, atm["kT"], x, jbar, np.stack([atm["bx"], atm["by"], atm["bz"]], -1))


def f_fine(tab, shape):
    f = np.zeros(tuple(shape) + (len(tab.rows),))
    f[..., tab.row0] = 1.0
    return f


def jacobi(atm, atom, tab, x, quad, src, n):
    bvec = np.stack([atm["bx"], atm["by"], atm["bz"]], -1)
    change = None
    for _ in range(n):
        jbar, lstar = formal_solve_lines(atm, atom, tab, x, quad)
        x, change = see_update(tab, atm["kT"], x, jbar, lstar, bvec, src)
    return x, change


def vcycle(levels, atom, tab, quad, x, src=None, l=0, npre=2, npost=4, ncoarse=8, order=1):
    """One V-cycle from level l (levels from ml.hierarchy) down to the coarsest."""
    from .mg import prolong, restrict
    lev = levels[l]
    f = f_fine(tab, lev.shape) if src is None else src
    if l == len(levels) - 1:
        x, _ = jacobi(lev.atm, atom, tab, x, quad, f, ncoarse)
        return x
    x, _ = jacobi(lev.atm, atom, tab, x, quad, f, npre)
    r = f - apply_A(lev.atm, atom, tab, x, quad)
    coarse = levels[l + 1]
    x_c0 = restrict(lev, x)
    f_c = apply_A(coarse.atm, atom, tab, x_c0, quad) + restrict(lev, r)
    x_c = vcycle(levels, atom, tab, quad, x_c0, f_c, l + 1, npre, npost, ncoarse, order)
    x = x + prolong(lev, x_c - x_c0, order)
    x, _ = jacobi(lev.atm, atom, tab, x, quad, f, npost)
    return x
