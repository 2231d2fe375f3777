"""Pins of the biquadratic (9-point) interpolation of the sweep (Sec. 3.1: the
upwind and downwind transfer coefficients and the upwind Stokes vector from the
9 nearest nodes of the neighbouring plane): exactness of the stencil on
tensor-product quadratics, partition of unity and node injection, the 3D = 1D
reduction for horizontally homogeneous boxes, equality with the bilinear sweep
where the stencil falls on nodes along one axis and the field is constant along
the other, and a smaller horizontal discretization error than the bilinear
stencil on grids that resolve the field."""
import numpy as np
import pytest

import oracle
import synth


def _prob(nx, ny, interp):
    a = synth.plane_parallel_box(nx, ny, 6)
    return oracle.Problem(a, 0, 1, 2, 2, interp=interp)


def test_biquadratic_stencil_is_exact_on_tensor_quadratics():
    p = _prob(16, 12, 2)
    rng = np.random.default_rng(4)
    for _ in range(200):
        xc, yc = rng.uniform(2.0, 13.0), rng.uniform(2.0, 9.0)        # no periodic wrap
        a, b = rng.normal(size=3), rng.normal(size=3)
        f = lambda x, y: (a[0] + a[1] * x + a[2] * x * x) * (b[0] + b[1] * y + b[2] * y * y) + 0.3 * x * y
        st = oracle.interp_weights(p, xc, yc, 2)
        assert len(st) == 9
        assert sum(w for _, _, w in st) == pytest.approx(1.0, abs=1e-14)
        assert sum(w * f(i, j) for i, j, w in st) == pytest.approx(f(xc, yc), rel=1e-11, abs=1e-11)
        # the bilinear stencil is exact only on bilinear functions
        g = lambda x, y: 1.0 + 2.0 * x - 0.5 * y + 0.25 * x * y
        assert sum(w * g(i, j) for i, j, w in oracle.interp_weights(p, xc, yc, 1)) == pytest.approx(g(xc, yc), rel=1e-12)
    # at a node: injection; the stencil wraps periodically
    st = [(i, j, w) for i, j, w in oracle.interp_weights(p, 15.0, 0.0, 2) if w != 0.0]
    assert st == [(15, 0, 1.0)]
    assert {(i, j) for i, j, _ in oracle.interp_weights(p, 15.4, 0.2, 2)} == {(i, j) for i in (14, 15, 0) for j in (11, 0, 1)}


def test_biquadratic_sweep_reduces_to_1d_for_homogeneous_layers():
    atm = synth.plane_parallel_box(6, 5, 20, modulation=0.0)
    rho = np.zeros((20, 5, 6, 1))
    rho[..., 0] = atm["bpl"]
    j1, l1 = oracle.formal_solve(oracle.Problem(atm, 0, 2, 4, 3, interp=1), rho)
    j2, l2 = oracle.formal_solve(oracle.Problem(atm, 0, 2, 4, 3, interp=2), rho)
    assert np.allclose(j2, j1, rtol=1e-12, atol=0)
    assert np.allclose(l2, l1, rtol=1e-12, atol=0)


def test_biquadratic_equals_bilinear_for_fields_along_the_other_axis():
    """Rays in the x-z plane (azimuths 0 and pi: no y offset) over a field that varies
    in y only: the y weights sit on nodes and the x interpolation of a constant is exact,
    for both stencils."""
    atm = synth.plane_parallel_box(6, 8, 12, modulation=0.0)
    y = np.arange(8) / 8.0
    atm["chi"] = atm["chi"] * (1.0 + 0.4 * np.sin(2 * np.pi * y))[None, :, None]
    rho = np.zeros((12, 8, 6, 1))
    rho[..., 0] = atm["bpl"]
    mu = np.array([0.3, 0.6, 0.8])
    chi = np.array([0.0, np.pi, 0.0])
    e1 = oracle.emergent(oracle.Problem(atm, 0, 1, 2, 3, interp=1), rho, mu, chi)
    e2 = oracle.emergent(oracle.Problem(atm, 0, 1, 2, 3, interp=2), rho, mu, chi)
    assert np.allclose(e2, e1, rtol=1e-12, atol=0)


def test_biquadratic_is_closer_to_the_fine_grid_solution_on_resolved_grids():
    def atm_x(nx):
        a = synth.plane_parallel_box(nx, 1, 8, modulation=0.0, tau_top=1e-2, tau_bot=1e2)
        x = np.arange(nx) / nx
        a["chi"] = a["chi"] * (1.0 + 0.5 * np.sin(2 * np.pi * x))[None, None, :]
        a["bpl"] = a["bpl"] * (1.0 + 0.3 * np.cos(2 * np.pi * x))[None, None, :]
        return a

    def jbar(nx, interp):
        a = atm_x(nx)
        rho = np.zeros((8, 1, nx, 1))
        rho[..., 0] = a["bpl"]
        j, _ = oracle.formal_solve(oracle.Problem(a, 0, 2, 4, 3, interp=interp), rho)
        return j[:, 0, :: nx // 8, 0]

    ref = jbar(128, 2)
    for nx in (32, 64):
        e1 = np.max(np.abs(jbar(nx, 1) / ref - 1))
        e2 = np.max(np.abs(jbar(nx, 2) / ref - 1))
        assert e2 < 0.75 * e1, (nx, e1, e2)


def test_reverse_mode_rejects_biquadratic():
    atm = synth.plane_parallel_box(4, 4, 6)
    p = oracle.Problem(atm, 0, 1, 2, 2, interp=2)
    rho = np.ones((6, 4, 4, 1))
    with pytest.raises(AssertionError):
        oracle.emergent_vjp(p, rho, np.array([0.5]), np.array([0.0]), np.ones((1, 2, 4, 4, 1)))
