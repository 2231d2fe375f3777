"""Pins of the orientation (K = 1) terms of the polarized multilevel atom
(oracle/mlpol.py, oracle/or_sweep.c): J^1_Q of the formal solution in a thick
homogeneous medium (I = S: J^1_Q = S^1_Q / 2 from the orthogonality of
T^1_Q(V, Omega) = sqrt(3/2) Omega_Q over the sphere); the dipole selection rules
(a J = 1 level with only M = +1 populated emits and absorbs 100 % circular
polarization along the quantization axis, none across it, and the photon the
emission M = +1 -> J = 0 creates has the opposite helicity to the one the
absorption m = +1 -> J = 0 destroys); and the J = 0 -> 1 two-level atom in zero
field, whose orientation scatters with W_1 = (w^(1))^2 = 1, S^1_Q = (1 - eps) J^1_Q."""
import numpy as np

import oracle
from oracle import ml, mlpol

from test_oracle_mlpol import _atom2, _eta_ratios, _sublevels


def _t1(mu, chi):
    st = np.sqrt(max(0.0, 1 - mu * mu))
    return np.array([np.sqrt(1.5) * mu, -np.sqrt(0.75) * st * np.cos(chi), -np.sqrt(0.75) * st * np.sin(chi)])


def _a1(t1, s):
    return t1[0] * s[0] + 2 * (t1[1] * s[1] + t1[2] * s[2])


def test_j1_of_a_thick_oriented_medium():
    nz, shape = 40, (40, 2, 2)
    atm = dict(nx=2, ny=2, nz=nz, lx=1.0, ly=1.0, z=np.arange(nz, dtype=np.float64), chi=np.full(shape, 300.0),
               eps=np.full(shape, 1e-2), bpl=np.full(shape, 0.9), vel=np.zeros(shape), bx=np.zeros(shape),
               by=np.zeros(shape), bz=np.zeros(shape), zeta=0.0, gbar=1.0, bcrit=25.0)
    s1 = np.array([0.07, -0.03, 0.05])
    atm["orient"] = np.broadcast_to(s1, shape + (3,)).copy()
    rho = np.zeros(shape + (6,))
    rho[..., 0] = 0.9
    p = oracle.Problem(atm, 1, 5, 16, 5, x_max=1.0)
    jkq, _, j1 = oracle.formal_solve(p, rho, with_j1=True)
    assert np.allclose(j1[8:32], s1 / 2, rtol=0, atol=1e-12)
    assert np.allclose(jkq[8:32, ..., 0], 0.9, rtol=1e-12)
    # no orientation source, no field: no circular polarization and no J^1
    atm.pop("orient")
    _, _, j1 = oracle.formal_solve(oracle.Problem(atm, 1, 2, 4, 3), rho, with_j1=True)
    assert np.max(np.abs(j1)) == 0.0


def test_orientation_follows_the_dipole_selection_rules():
    # emission J_u = 1 (only M = +1) -> J_l = 0: S_V = +-S_I along z, S_V = 0 along x
    tab = mlpol.Tables(_atom2(0, 1))
    x = _sublevels(tab, 0, [1.0]) + _sublevels(tab, 1, [0.0, 0.0, 0.2])
    src = mlpol.line_source_multipoles(tab, x)[0]
    ori = mlpol.line_orientation_multipoles(tab, x)[0]
    t = oracle.tkq(1.0, 0.0)
    SI = t[0, 0] * src[0] + t[0, 1] * src[1] + 2 * (t[0, 2] * src[2] + t[0, 3] * src[3]) + 2 * (t[0, 4] * src[4] + t[0, 5] * src[5])
    SV = _a1(_t1(1.0, 0.0), ori)
    assert abs(abs(SV) - SI) < 1e-12 * SI and SI > 0
    assert abs(_a1(_t1(0.0, 0.4), ori)) < 1e-14 * SI
    # absorption J_l = 1 (only m = +1) -> J_u = 0: eta_V = +-eta_I along z, 0 along x
    tab = mlpol.Tables(_atom2(1, 0))
    x = _sublevels(tab, 0, [0.0, 0.0, 1.0])                 # no upper population: absorption alone
    d2 = mlpol.line_dichroism(tab, x, 0)
    d1 = mlpol.line_dichroism_orientation(tab, x, 0)
    eI = _eta_ratios(d2, 1.0, 0.0)[0]
    eV = _a1(_t1(1.0, 0.0), d1)
    assert abs(abs(eV) - eI) < 1e-12 * eI and eI > 0
    assert abs(_a1(_t1(0.0, 1.3), d1)) < 1e-14
    # opposite helicities: the M = +1 -> 0 photon is emitted, the m = +1 -> 0 photon absorbed
    assert np.sign(SV) == -np.sign(eV)


def test_j0_to_j1_atom_scatters_orientation_with_unit_polarizability():
    at = _atom2(0, 1)
    tab = mlpol.Tables(at, stimulated=False)
    rng = np.random.default_rng(8)
    n = 4
    kT = rng.uniform(0.4, 0.6, n)
    jr = np.zeros((n, 1, 9))
    jr[..., 0] = rng.uniform(0.5, 1.5, size=(n, 1))
    jr[..., 1:4] = rng.normal(size=(n, 1, 3)) * 0.1
    jr[..., 4:9] = rng.normal(size=(n, 1, 5)) * 0.1
    x = tab.solve(tab.matrix(kT, jr, np.zeros((n, 3))))
    ori = mlpol.line_orientation_multipoles(tab, x)[:, 0]
    pops = tab.populations(x)
    Sw = pops[:, 1] / 3 / pops[:, 0]                 # the line source function without stimulated emission
    S = ml.source_function(at, pops)[:, 0]
    cul, _ = ml.collision_rates(at, kT)
    eps = cul[0] / (at["A"][0] + cul[0])
    # S^1_Q with the source function Sw of the two-level atom: (1 - eps) J^1_Q
    want = (1 - eps) * jr[:, 0, 1:4]
    got = ori * (Sw / S)[:, None]
    assert np.allclose(got, want, rtol=1e-10, atol=1e-13)
