"""Pins of the oracle's weak-field Zeeman terms (the Stokes V of the two-level
atom, Sec. 2 and Sec. 3.3 with the propagation matrix of Eq. 8).

The model takes the first-order Zeeman term of a line with a Doppler profile:
eta_V = 2 gbar zeta (x - s) (B.Omega) eta_I and eps_V = S^0_0 eta_V, i.e.
eta_V = -gbar zeta (B.Omega) d(eta_I)/dx and, while the source function is
unpolarized (S^2_Q = 0, so S_I = S^0_0), eps_V = -gbar zeta (B.Omega) d(eps_I)/dx.
Two consequences are independent of how the oracle is written:

* reversing the field reverses Stokes V and leaves I, Q and U unchanged (the
  transfer equation is invariant under V -> -V, eta_V -> -eta_V, eps_V -> -eps_V);
* to first order in the splitting, V = -gbar zeta (B.Omega) dI/dx along every ray:
  differentiating the transfer equation for I in x gives the equation for V with
  the same (zero) boundary value. This is the weak-field relation between V and
  the intensity derivative; the discrete solutions obey it up to the formal
  solver's discretization error, which must shrink as the grid is refined.

A flipped sign of eps_V against eta_V, a factor 2 in either, a field component
or direction cosine taken from the wrong axis, or V coupled with the wrong sign
into the 4x4 step fails the second pin.
"""
import numpy as np

import oracle
import synth


def _random_pol(nx, ny, nz, seed):
    atm = synth.random_box(nx, ny, nz, seed=seed)
    atm["zeta"] = 1e-3
    return atm


def test_field_reversal_reverses_stokes_v_only():
    atm = _random_pol(6, 5, 8, seed=21)
    p = oracle.Problem(atm, oracle.MODEL_HANLE, 2, 4, 7)
    rng = np.random.default_rng(22)
    rho = np.zeros(p.shape + (6,))
    rho[..., 0] = atm["bpl"]
    rho[..., 1:] = 0.05 * rho[..., :1] * rng.normal(size=p.shape + (5,))
    mu = np.array([1.0, 0.5, 0.5, 0.3])
    az = np.array([0.0, 0.7, 3.9, 2.0])
    out = oracle.emergent(p, rho, mu, az)
    rev = dict(atm)
    rev["bx"], rev["by"], rev["bz"] = -atm["bx"], -atm["by"], -atm["bz"]
    out_r = oracle.emergent(oracle.Problem(rev, oracle.MODEL_HANLE, 2, 4, 7), rho, mu, az)
    scale = np.max(np.abs(out[..., 0]))
    assert np.max(np.abs(out_r[..., :3] - out[..., :3])) <= 1e-14 * scale
    assert np.max(np.abs(out_r[..., 3] + out[..., 3])) <= 1e-14 * scale
    assert np.max(np.abs(out[..., 3])) > 1e-4 * scale       # V is not trivially zero


def _layered(nz, b, mu_dirs):
    """Horizontally homogeneous box (2x2 columns): exponential opacity over log-spaced
    optical depths 1e-3..1e2, a smooth unpolarized source function, a uniform field."""
    z = synth.log_tau_heights(nz, tau_top=1e-3, tau_bot=1e2)
    tau = np.exp(-z / synth.H_KM)
    shape = (nz, 2, 2)
    atm = dict(nx=2, ny=2, nz=nz, lx=800.0, ly=800.0, z=z,
               chi=np.broadcast_to(synth.exponential_opacity(z)[:, None, None], shape).copy(),
               eps=np.full(shape, 1e-2), bpl=np.full(shape, 1.0), vel=np.zeros(shape),
               bx=np.full(shape, b[0]), by=np.full(shape, b[1]), bz=np.full(shape, b[2]),
               zeta=1e-6, gbar=1.0, bcrit=25.0)
    S = 1.0 + 0.6 * np.tanh(np.log10(tau))                  # smooth, monotonic in depth
    rho = np.zeros(shape + (6,))
    rho[..., 0] = S[:, None, None]
    return atm, rho


def test_weak_field_stokes_v_is_the_intensity_derivative():
    b = np.array([30.0, -20.0, 40.0])
    mu = np.array([1.0, 0.5, 0.5])
    az = np.array([0.0, 0.3, 2.5])
    n_nu, dv = 15, 1e-4
    errs = []
    for nz in (24, 48, 96):
        atm, rho = _layered(nz, b, mu)
        p = oracle.Problem(atm, oracle.MODEL_HANLE, 2, 4, n_nu)
        out = oracle.emergent(p, rho, mu, az)
        # dI/dx from a uniform velocity shift: the profiles depend on x - v mu
        shifted = []
        for sgn in (1.0, -1.0):
            a = dict(atm)
            a["vel"] = np.full(atm["chi"].shape, sgn * dv)
            shifted.append(oracle.emergent(oracle.Problem(a, oracle.MODEL_HANLE, 2, 4, n_nu), rho, mu, az))
        dIdv = (shifted[0][..., 0] - shifted[1][..., 0]) / (2 * dv)
        st = np.sqrt(1.0 - mu * mu)
        bdotomega = b[0] * st * np.cos(az) + b[1] * st * np.sin(az) + b[2] * mu
        dIdx = -dIdv / mu[:, None, None, None]
        want = -atm["gbar"] * atm["zeta"] * bdotomega[:, None, None, None] * dIdx
        V = out[..., 3]
        scale = np.max(np.abs(want), axis=(1, 2, 3), keepdims=True)
        errs.append(float(np.max(np.abs(V - want) / scale)))
    # discretization error of the formal solver: shrinks with refinement, and is
    # small at 96 planes over five decades of optical depth
    print("weak-field V errors", errs)
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1], errs
    assert errs[2] < 2e-3, errs
