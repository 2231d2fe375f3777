"""Pins of the oracle's short characteristics on the first cell face they cross
(Sec. 3.1: M and P may lie on a vertical plane of the grid), `sc_faces=1`.

* S linear in height with the matching lower boundary: the exact I = a + b tau_v
  + b |mu|/phi is linear in height and uniform horizontally, so the bilinear face
  stencil (horizontal position, height between two planes) and BESSER are exact
  for every ray, the grazing ones whose upwind face is vertical included (their
  face's upper nodes lie on the point's own plane: the periodic chain of the plane
  must close on the exact solution);
* a horizontally homogeneous slab with a boundary: every plane stays uniform
  (a wrong wrap or order of the in-plane chain breaks the uniformity);
* opaque medium with constant S: I = S;
* rays whose offset over every layer stays within one cell: identical to the
  sweep on horizontal planes (the same stencil).
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _uniform_atm(nx, ny, nz, chi=1.0, dz=1.0, dx=1.0, bpl=1.0):
    shape = (nz, ny, nx)
    return dict(nx=nx, ny=ny, nz=nz, lx=nx * dx, ly=ny * dx, z=np.arange(nz) * dz,
                chi=np.full(shape, chi), eps=np.full(shape, 0.1), bpl=np.full(shape, bpl),
                vel=np.zeros(shape), zeta=3.5e-4, gbar=1.0, bcrit=25.0)


def _vertical(p, m, dz, dx):
    mu, chi, _ = oracle.rays(p)
    t = math.sqrt(1 - mu[m] ** 2) / abs(mu[m])
    return dz * t * max(abs(math.cos(chi[m])), abs(math.sin(chi[m]))) / dx > 1.0


def test_linear_source_is_exact_on_vertical_faces():
    nx, ny, nz, dz = 4, 5, 24, 0.7
    atm = _uniform_atm(nx, ny, nz, chi=1.5, dz=dz)
    z = atm["z"]
    tau_v = 1.5 * (z[-1] - z)
    a0, b0 = 0.3, 0.8
    p = oracle.Problem(atm, 0, 3, 6, 5, sc_faces=1)
    mu, _, _ = oracle.rays(p)
    xf, _ = oracle.freqs(5, 4.0)
    rho = np.broadcast_to((a0 + b0 * tau_v)[:, None, None, None], p.shape + (1,)).copy()
    nvert = 0
    for m in range(18):                          # upward rays
        for j in [1, 2]:
            ph = math.exp(-xf[j] ** 2)
            exact = a0 + b0 * tau_v + b0 * abs(mu[m]) / ph
            atm2 = dict(atm)
            atm2["bpl"] = np.broadcast_to(exact[:, None, None], p.shape).copy()
            p2 = oracle.Problem(atm2, 0, 3, 6, 5, sc_faces=1)
            I, _ = oracle.sweep_ray(p2, rho, m, j)
            assert np.allclose(I[..., 0], exact[:, None, None], rtol=1e-12), (m, j)
        nvert += _vertical(p, m, dz, 1.0)
    assert nvert >= 6                            # grazing rays do meet vertical faces


def test_homogeneous_slab_stays_uniform_in_every_plane():
    atm = _uniform_atm(5, 4, 12, chi=0.8, dz=1.2, bpl=1.0)
    p = oracle.Problem(atm, 0, 3, 8, 3, sc_faces=1)
    rho = np.full(p.shape + (1,), 0.4)           # constant S below the boundary value
    for m in [0, 3, 9, 20, 30]:
        for j in [0, 1]:
            I, ls = oracle.sweep_ray(p, rho, m, j)
            spread = np.max(np.abs(I[..., 0] - I[:, :1, :1, 0]), axis=(1, 2))
            assert np.max(spread) < 1e-13, (m, j)
            assert np.all(np.isfinite(ls))


def test_opaque_medium_gives_I_equal_S():
    atm = _uniform_atm(3, 3, 30, chi=200.0, dz=1.0, dx=0.05, bpl=0.7)
    p = oracle.Problem(atm, 0, 3, 8, 5, x_max=1.0, sc_faces=1)
    rho = np.full(p.shape + (1,), 0.7)
    jkq, ls = oracle.formal_solve(p, rho)
    assert np.allclose(jkq[:20, ..., 0], 0.7, rtol=1e-12)


def test_short_offsets_equal_the_plane_sweep():
    rng = np.random.default_rng(3)
    nx, ny, nz = 4, 3, 10
    atm = _uniform_atm(nx, ny, nz, dz=0.1, dx=5.0)
    atm["chi"] = np.exp(rng.normal(size=(nz, ny, nx)))
    atm["vel"] = 0.5 * rng.normal(size=(nz, ny, nx))
    rho = rng.uniform(0.5, 1.5, (nz, ny, nx, 1))
    a = oracle.Problem(atm, 0, 2, 4, 3)
    b = oracle.Problem(atm, 0, 2, 4, 3, sc_faces=1)
    mu, _, _ = oracle.rays(a)
    assert all(not _vertical(a, m, 0.1, 5.0) for m in range(len(mu)))
    ja, la = oracle.formal_solve(a, rho)
    jb, lb = oracle.formal_solve(b, rho)
    assert np.array_equal(ja, jb) and np.array_equal(la, lb)


def test_faces_option_is_checked():
    atm = _uniform_atm(3, 3, 6)
    p = oracle.Problem(atm, 0, 2, 4, 3, interp=2, sc_faces=1)
    with pytest.raises(AssertionError):
        oracle.formal_solve(p, np.ones(p.shape + (1,)))


def _smooth_box(n, size=4.0):
    """a box smooth in x and height, periodic in x and y (functions of x and z only)"""
    nx = ny = nz = n
    x = (np.arange(nx) + 0.0) * size / nx
    z = np.arange(nz) * size / (nz - 1)
    X = np.broadcast_to(x[None, None, :], (nz, ny, nx))
    Z = np.broadcast_to(z[:, None, None], (nz, ny, nx))
    atm = dict(nx=nx, ny=ny, nz=nz, lx=size, ly=size, z=z,
               chi=(1.0 + 0.5 * np.sin(2 * np.pi * X / size)) * np.exp(-0.3 * Z),
               eps=np.full((nz, ny, nx), 0.1), bpl=np.full((nz, ny, nx), 1.0),
               vel=np.zeros((nz, ny, nx)), zeta=3.5e-4, gbar=1.0, bcrit=25.0)
    S = 1.0 + 0.3 * np.cos(2 * np.pi * X / size) + 0.2 * Z
    return atm, np.ascontiguousarray(S[..., None])


def test_faces_and_planes_converge_to_the_same_field():
    """Both placements of M and P are consistent discretizations of the same transfer
    equation: for grazing rays, whose upwind points lie on vertical faces, the two
    fields approach each other as the grid is refined (a wrong horizontal offset,
    face or order would leave an O(1) difference)."""
    diffs = []
    for n in (8, 16, 32):
        atm, S = _smooth_box(n)
        a = oracle.Problem(atm, 0, 3, 4, 3)
        b = oracle.Problem(atm, 0, 3, 4, 3, sc_faces=1)
        mu, _, _ = oracle.rays(a)
        d = 0.0
        for m in range(12):                          # upward rays, the grazing ones first
            if not _vertical(a, m, atm["z"][1] - atm["z"][0], atm["lx"] / n):
                continue
            Ia, _ = oracle.sweep_ray(a, S, m, 1)
            Ib, _ = oracle.sweep_ray(b, S, m, 1)
            top = slice(n // 2, n)                   # away from the lower boundary layer
            d = max(d, np.max(np.abs(Ia[top, ..., 0] - Ib[top, ..., 0])))
        diffs.append(d)
    assert diffs[0] > 0
    assert diffs[2] < 0.5 * diffs[1] < 0.25 * diffs[0], diffs


def test_multilevel_lines_take_the_face_option():
    """The lines of the multilevel atom are two-level problems each (Sec. 2), so the
    face placement applies per line: with short offsets every line's sums equal the
    plane sweep's exactly; with grazing offsets they differ."""
    from oracle import ml
    atom = synth.multilevel_atom(seed=4, eps_range=(1e-3, 1e-1))
    quad = (2, 4, 3)
    wide = synth.multilevel_box(4, 3, 8, seed=5, tau_top=1e-2, tau_bot=1e1)
    wide["lx"], wide["ly"] = 1e5, 1e5              # cells far wider than any offset
    pops = ml.lte_populations(atom, wide["kT"])
    ja, la = ml.formal_solve_lines(wide, atom, pops, quad)
    jb, lb = ml.formal_solve_lines(wide, atom, pops, quad, sc_faces=1)
    assert np.array_equal(ja, jb) and np.array_equal(la, lb)
    narrow = synth.multilevel_box(4, 3, 8, seed=5, tau_top=1e-2, tau_bot=1e1)
    narrow["lx"], narrow["ly"] = 40.0, 30.0        # 10 km cells under ~100 km layers
    ja, _ = ml.formal_solve_lines(narrow, atom, pops, quad)
    jb, _ = ml.formal_solve_lines(narrow, atom, pops, quad, sc_faces=1)
    assert np.max(np.abs(jb / ja - 1)) > 1e-3
