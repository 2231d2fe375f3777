"""Plain FP64 CPU oracle of the PORTA formal-solver hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA
library: the C sources in this directory restate the paper (Stepan &
Trujillo Bueno 2013, arXiv:1307.4217) directly, one plain loop nest in
double precision.

Parity pins: see ``tests/test_oracle_*.py``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_SRCS = ["or_quad.c", "or_besser.c", "or_sweep.c", "or_see.c", "oracle.h", "or_common.h"]

MODEL_UNPOL = 0
MODEL_HANLE = 1
BESSER = 0
DELOPAR = 1
LINEAR = 2
BEZIER_FB = 3
CBEZIER = 4


def build(force=False):
    """Compile liboracle.so with gcc (no fast-math, no FMA contraction)."""
    if not force and os.path.exists(_LIB):
        newest = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SRCS)
        if os.path.getmtime(_LIB) >= newest:
            return _LIB
    subprocess.run(["sh", os.path.join(_HERE, "build.sh")], check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("z", ctypes.c_void_p),
        ("model", ctypes.c_int),
        ("chi", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("bpl", ctypes.c_void_p),
        ("vel", ctypes.c_void_p), ("bx", ctypes.c_void_p), ("by", ctypes.c_void_p),
        ("bz", ctypes.c_void_p),
        ("zeta", ctypes.c_double), ("gbar", ctypes.c_double), ("bcrit", ctypes.c_double),
        ("n_mu", ctypes.c_int), ("n_chi", ctypes.c_int), ("n_nu", ctypes.c_int),
        ("x_max", ctypes.c_double),
        ("method", ctypes.c_int),
        ("dich", ctypes.c_void_p),
        ("interp", ctypes.c_int),
        ("kexpl", ctypes.c_void_p),
        ("sexpl", ctypes.c_void_p),
        ("orient", ctypes.c_void_p),
        ("dich1", ctypes.c_void_p),
        ("j1", ctypes.c_void_p),
        ("sc_faces", ctypes.c_int),
    ]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def _declare(L):
    sig = {
        "or_gauss_legendre01": (_I, [_I, _P, _P]),
        "or_rays": (_I, [_P, _P, _P, _P]),
        "or_freqs": (_I, [_I, _D, _P, _P]),
        "or_tkq": (None, [_D, _D, _P]),
        "or_coeffs": (None, [_D, _P]),
        "or_control_point": (_D, [_D, _D, _D, _D, _D, _I, _I]),
        "or_interp_weights": (_I, [_P, _D, _D, _I, _P, _P, _P]),
        "or_solve_1d": (_I, [_I, _P, _P, _D, _I, _P]),
        "or_step": (_I, [_I, _P, _P, _P, _P, _P, _D, _P, _D, _D, _I, _I, _P, _P]),
        "or_hanle_solve": (_I, [_D, _D, _D, _D, _P, _P]),
        "or_see_update": (_I, [_P, _P, _P, _P, _P]),
        "or_sweep_ray": (_I, [_P, _P, _I, _I, _P, _P]),
        "or_formal_solve": (_I, [_P, _P, _P, _P]),
        "or_formal_solve_part": (_I, [_P, _P, _I, _I, _I, _I, _P, _P]),
        "or_emergent": (_I, [_P, _P, _I, _P, _P, _P]),
        "or_emergent_vjp": (_I, [_P, _P, _I, _P, _P, _P, _P, _P, _P]),
        "or_coeffs_deriv": (None, [_D, _P, _P]),
        "or_control_point_vjp": (None, [_D, _D, _D, _D, _D, _I, _I, _D, _P]),
        "or_step_vjp": (_I, [_I, _P, _P, _P, _P, _P, _D, _P, _D, _D, _I, _I, _P,
                             _P, _P, _P, _P, _P, _P, _P]),
        "or_see_apply": (_I, [_P, _P, _P, _P]),
        "or_see_update_src": (_I, [_P, _P, _P, _P, _P, _P]),
        "or_see_update_vjp": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "or_jkq_vjp": (_I, [_P, _P, _P, _P, _P, _P, _P]),
        "or_emergent_vjp_rho": (_I, [_P, _P, _I, _P, _P, _P, _P, _P, _P]),
        "or_flops_reset": (None, [_I]),
        "or_flops_get": (ctypes.c_longlong, []),
        "or_nray": (_I, [_P]),
        "or_branch_sig_reset": (None, [_I]),
        "or_branch_sig_get": (ctypes.c_ulonglong, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data if a is not None else None


def ns_of(model):
    return 1 if model == MODEL_UNPOL else 4


def nl_of(model):
    return 1 if model == MODEL_UNPOL else 6


def nj_of(model):
    return 1 if model == MODEL_UNPOL else 6


class Problem:
    """Holds the arrays referenced by the C problem struct (keeps them alive).

    ``atm`` is a dict with keys nx, ny, nz, lx, ly, z, chi, eps, bpl, vel and,
    for the polarized model, bx, by, bz (per-voxel arrays in (nz, ny, nx) order),
    plus the atomic constants zeta, gbar, bcrit.
    """

    def __init__(self, atm, model, n_mu, n_chi, n_nu, x_max=4.0, method=BESSER, interp=1, sc_faces=0):
        self.model = model
        self.shape = (atm["nz"], atm["ny"], atm["nx"])
        self.nvox = int(np.prod(self.shape))
        self._keep = {}
        for k in ("z", "chi", "eps", "bpl", "vel", "bx", "by", "bz"):
            v = atm.get(k)
            self._keep[k] = _f64(v).ravel() if v is not None else None
        s = _Problem()
        s.nx, s.ny, s.nz = atm["nx"], atm["ny"], atm["nz"]
        s.lx, s.ly = float(atm["lx"]), float(atm["ly"])
        for k in ("z", "chi", "eps", "bpl", "vel", "bx", "by", "bz"):
            setattr(s, k, _ptr(self._keep[k]))
        s.model = model
        s.zeta = float(atm.get("zeta", 0.0))
        s.gbar = float(atm.get("gbar", 1.0))
        s.bcrit = float(atm.get("bcrit", 25.0))
        s.n_mu, s.n_chi, s.n_nu = n_mu, n_chi, n_nu
        s.x_max = float(x_max)
        s.method = method
        d = atm.get("dich")
        self._keep["dich"] = _f64(d).ravel() if d is not None else None
        s.dich = _ptr(self._keep["dich"])
        s.interp = int(interp)          # 1 bilinear, 2 biquadratic (Sec. 3.1)
        # 0: M and P on the next horizontal planes; 1: on the first cell face the short
        # characteristic crosses, vertical faces included (Sec. 3.1; forward sweeps only)
        s.sc_faces = int(sc_faces)
        # explicit medium: atm["kexpl"] (6, nz, ny, nx) = (eta_Q, eta_U, eta_V, rho_Q, rho_U,
        # rho_V) / eta_I and atm["sexpl"] (4, nz, ny, nx) = S, per voxel (polarized model)
        for k in ("kexpl", "sexpl"):
            v = atm.get(k)
            self._keep[k] = _f64(v).ravel() if v is not None else None
            setattr(s, k, _ptr(self._keep[k]))
        # orientation terms of a polarized line: atm["orient"] (nz, ny, nx, 3) = S^1_Q and
        # atm["dich1"] (nz, ny, nx, 3) = D^1_Q in the layout (X10, Re X11, Im X11)
        for k in ("orient", "dich1"):
            v = atm.get(k)
            self._keep[k] = _f64(v).ravel() if v is not None else None
            setattr(s, k, _ptr(self._keep[k]))
        s.j1 = None
        self.interp = int(interp)
        self.s = s
        self.nray = 2 * n_mu * n_chi
        self.n_nu = n_nu

    @property
    def ref(self):
        return ctypes.byref(self.s)


def gauss_legendre01(n):
    x = np.zeros(n); w = np.zeros(n)
    assert lib().or_gauss_legendre01(n, _ptr(x), _ptr(w)) == 0
    return x, w


def rays(prob):
    n = prob.nray
    mu, chi, w = np.zeros(n), np.zeros(n), np.zeros(n)
    assert lib().or_rays(prob.ref, _ptr(mu), _ptr(chi), _ptr(w)) == 0
    return mu, chi, w


def freqs(n_nu, x_max):
    x, w = np.zeros(n_nu), np.zeros(n_nu)
    assert lib().or_freqs(n_nu, float(x_max), _ptr(x), _ptr(w)) == 0
    return x, w


def tkq(mu, chi):
    t = np.zeros(18)
    lib().or_tkq(float(mu), float(chi), _ptr(t))
    return t.reshape(3, 6)


def coeffs(tau):
    c = np.zeros(6)
    lib().or_coeffs(float(tau), _ptr(c))
    return c


def interp_weights(prob, xc, yc, order):
    """nodes (i, j) and weights of the sweep's periodic interpolation stencil at cell
    coordinates (xc, yc): order 1 bilinear, 2 biquadratic"""
    ii = (ctypes.c_int * 9)()
    jj = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    n = lib().or_interp_weights(prob.ref, float(xc), float(yc), int(order), ii, jj, w)
    return [(ii[k], jj[k], w[k]) for k in range(n)]


def control_point(yM, yO, yP, hM, hP, has_p=True, method=BESSER):
    return lib().or_control_point(yM, yO, yP, hM, hP, int(has_p), method)


def solve_1d(tau, S, I0, method=BESSER):
    tau = _f64(tau); S = _f64(S)
    out = np.zeros_like(tau)
    assert lib().or_solve_1d(len(tau), _ptr(tau), _ptr(S), float(I0), method, _ptr(out)) == 0
    return out


# ---- the one-ray sigmoid benchmark of Sec. 3.4 (Eqs. 15-18) ----
def sigmoid(a, d, z):
    """Eq. 16: sigma(a, d, z) = 1 / (1 + exp(-a (z - d)))."""
    return 1.0 / (1.0 + np.exp(-a * (np.asarray(z, dtype=np.float64) - d)))


def sigmoid_source(z):
    """Eq. 15: S(z) = sigma(2, -5, z) sigma(-2, 5, z) (constant opacity, z = tau)."""
    return sigmoid(2.0, -5.0, z) * sigmoid(-2.0, 5.0, z)


def sigmoid_exact(z):
    """Eq. 17: the analytic intensity towards +z for I(-inf) = 0."""
    z = np.asarray(z, dtype=np.float64)
    return np.exp(15.0 - z) / (np.exp(20.0) - 1.0) * (np.exp(10.0) * np.arctan(np.exp(z - 5.0))
                                                      - np.arctan(np.exp(z + 5.0)))


def sigmoid_grid(dtau, shift=0.0):
    """Nodes z_k = -12 + shift + k dtau within [-12, 12] (shift in [0, dtau))."""
    n = int(np.floor((24.0 - shift) / dtau + 1e-9)) + 1
    return -12.0 + shift + dtau * np.arange(n)


def sigmoid_error(dtau, method=BESSER, shift=0.0):
    """E(dtau) (Eq. 18): max over the nodes of |I - I_a| / I_a, starting from the
    exact intensity at the first node (the paper's boundary value at z = -12)."""
    z = sigmoid_grid(dtau, shift)
    ia = sigmoid_exact(z)
    I = solve_1d(z - z[0], sigmoid_source(z), ia[0], method)
    return float(np.max(np.abs((I - ia) / ia)))


def step(ns, IM, etaM, epsM, etaO, epsO, etaP_I, epsP, dsM, dsP, has_p=True, method=BESSER):
    a = [_f64(x) for x in (IM, etaM, epsM, etaO, epsO, epsP)]
    IO = np.zeros(ns); ls = np.zeros(1)
    rc = lib().or_step(ns, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]), float(etaP_I),
                       _ptr(a[5]), float(dsM), float(dsP), int(has_p), method, _ptr(IO), _ptr(ls))
    assert rc == 0
    return IO, ls[0]


def hanle_solve(gamma, b, rhs6):
    rhs6 = _f64(rhs6); out = np.zeros(6)
    assert lib().or_hanle_solve(float(gamma), float(b[0]), float(b[1]), float(b[2]), _ptr(rhs6), _ptr(out)) == 0
    return out


def formal_solve(prob, rho, rays_range=None, freq_range=None, with_j1=False):
    """J^K_Q (K = 0, 2) and Lambda-bar*; with_j1 also J^1_Q (layout J10, Re J11, Im J11,
    from Stokes V; polarized model)."""
    rho = _f64(rho).ravel()
    assert rho.size == prob.nvox * nl_of(prob.model)
    jkq = np.zeros(prob.nvox * nj_of(prob.model)); ls = np.zeros(prob.nvox)
    m0, m1 = rays_range if rays_range else (0, prob.nray)
    j0, j1 = freq_range if freq_range else (0, prob.n_nu)
    jo = np.zeros(prob.nvox * 3) if with_j1 else None
    prob.s.j1 = _ptr(jo) if with_j1 else None
    rc = lib().or_formal_solve_part(prob.ref, _ptr(rho), m0, m1, j0, j1, _ptr(jkq), _ptr(ls))
    prob.s.j1 = None
    assert rc == 0, rc
    out = (jkq.reshape(prob.shape + (nj_of(prob.model),)), ls.reshape(prob.shape))
    return out + (jo.reshape(prob.shape + (3,)),) if with_j1 else out


def sweep_ray(prob, rho, m, j):
    rho = _f64(rho).ravel()
    ns = ns_of(prob.model)
    I = np.zeros(prob.nvox * ns); ls = np.zeros(prob.nvox)
    assert lib().or_sweep_ray(prob.ref, _ptr(rho), m, j, _ptr(I), _ptr(ls)) == 0
    return I.reshape(prob.shape + (ns,)), ls.reshape(prob.shape)


def see_update(prob, jkq, lstar, rho):
    jkq = _f64(jkq).ravel(); lstar = _f64(lstar).ravel()
    rho = _f64(rho).copy().ravel()
    mc = np.zeros(1)
    assert lib().or_see_update(prob.ref, _ptr(jkq), _ptr(lstar), _ptr(rho), _ptr(mc)) == 0
    return rho.reshape(prob.shape + (nl_of(prob.model),)), float(mc[0])


def see_apply(prob, jkq, rho):
    """A(S) of the statistical-equilibrium equations written as A(S) = f."""
    jkq = _f64(jkq).ravel(); rho = _f64(rho).ravel()
    out = np.zeros_like(rho)
    assert lib().or_see_apply(prob.ref, _ptr(jkq), _ptr(rho), _ptr(out)) == 0
    return out.reshape(prob.shape + (nl_of(prob.model),))


def see_update_src(prob, jkq, lstar, rho, src=None):
    """Jacobi update of A(S) = src (src None: the two-level problem, src = eps B delta_K0)."""
    jkq = _f64(jkq).ravel(); lstar = _f64(lstar).ravel()
    rho = _f64(rho).copy().ravel()
    s = _f64(src).ravel() if src is not None else None
    mc = np.zeros(1)
    assert lib().or_see_update_src(prob.ref, _ptr(jkq), _ptr(lstar), _ptr(s), _ptr(rho), _ptr(mc)) == 0
    return rho.reshape(prob.shape + (nl_of(prob.model),)), float(mc[0])


def emergent(prob, rho, mu, chi):
    rho = _f64(rho).ravel()
    mu = _f64(mu); chi = _f64(chi)
    ns = ns_of(prob.model)
    nz, ny, nx = prob.shape
    out = np.zeros(len(mu) * prob.n_nu * ny * nx * ns)
    assert lib().or_emergent(prob.ref, _ptr(rho), len(mu), _ptr(mu), _ptr(chi), _ptr(out)) == 0
    return out.reshape(len(mu), prob.n_nu, ny, nx, ns)


def coeffs_deriv(tau):
    """d/dtau of (e^-tau, psi'_M, psi'_O, w_M, w_O, w_C)."""
    c = coeffs(tau)
    d = np.zeros(6)
    lib().or_coeffs_deriv(float(tau), _ptr(c), _ptr(d))
    return d


def control_point_vjp(yM, yO, yP, hM, hP, has_p=True, method=BESSER, gc=1.0):
    """Gradient of the control point with respect to (yM, yO, yP, hM, hP), times gc
    (BESSER and DELOPAR)."""
    if method not in (BESSER, DELOPAR):
        raise ValueError("reverse mode is defined for BESSER and DELOPAR")
    g = np.zeros(5)
    lib().or_control_point_vjp(yM, yO, yP, hM, hP, int(has_p), method, float(gc), _ptr(g))
    return g


def step_vjp(ns, IM, etaM, epsM, etaO, epsO, etaP_I, epsP, dsM, dsP, gIO, has_p=True, method=BESSER):
    """Reverse mode of ``step``: gradients with respect to (IM, etaM[7], epsM, etaO[7], epsO, etaP_I, epsP)."""
    a = [_f64(x) for x in (IM, etaM, epsM, etaO, epsO, epsP, gIO)]
    out = dict(IM=np.zeros(ns), etaM=np.zeros(7), epsM=np.zeros(ns), etaO=np.zeros(7),
               epsO=np.zeros(ns), etaP=np.zeros(1), epsP=np.zeros(ns))
    rc = lib().or_step_vjp(ns, _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]), float(etaP_I),
                           _ptr(a[5]), float(dsM), float(dsP), int(has_p), method, _ptr(a[6]),
                           *[_ptr(out[k]) for k in ("IM", "etaM", "epsM", "etaO", "epsO", "etaP", "epsP")])
    assert rc == 0
    out["etaP"] = float(out["etaP"][0])
    return out


def emergent_vjp(prob, rho, mu, chi, gout):
    """Adjoint of ``emergent``: gradients of sum(gout * emergent(...)) with respect to per-voxel
    chi, e = chi S^0_0 (multipole ratios S^K_Q / S^0_0 fixed) and B (3, nz, ny, nx)."""
    rho = _f64(rho).ravel()
    mu = _f64(mu); chi = _f64(chi)
    ns = ns_of(prob.model)
    nz, ny, nx = prob.shape
    gout = _f64(gout).ravel()
    assert gout.size == len(mu) * prob.n_nu * ny * nx * ns
    g_chi = np.zeros(prob.nvox); g_e = np.zeros(prob.nvox); g_b = np.zeros(3 * prob.nvox)
    rc = lib().or_emergent_vjp(prob.ref, _ptr(rho), len(mu), _ptr(mu), _ptr(chi), _ptr(gout),
                               _ptr(g_chi), _ptr(g_e), _ptr(g_b))
    assert rc == 0, rc
    return g_chi.reshape(prob.shape), g_e.reshape(prob.shape), g_b.reshape((3,) + prob.shape)


def see_update_vjp(prob, jkq, lstar, rho, g, src=None):
    """Reverse mode of see_update_src: (dL/drho explicit, dL/dJ, dL/dLambda*, dL/dsrc^0_0, dL/dB)."""
    nl, nj = nl_of(prob.model), nj_of(prob.model)
    a = [_f64(x).ravel() for x in (jkq, lstar)]
    sr = _f64(src).ravel() if src is not None else None
    b = [_f64(x).ravel() for x in (rho, g)]
    out = dict(rho=np.zeros(prob.nvox * nl), jkq=np.zeros(prob.nvox * nj), lstar=np.zeros(prob.nvox),
               eb=np.zeros(prob.nvox), b=np.zeros(3 * prob.nvox))
    rc = lib().or_see_update_vjp(prob.ref, _ptr(a[0]), _ptr(a[1]), _ptr(sr), _ptr(b[0]), _ptr(b[1]),
                                 *[_ptr(out[k]) for k in ("rho", "jkq", "lstar", "eb", "b")])
    assert rc == 0
    sh = prob.shape
    return (out["rho"].reshape(sh + (nl,)), out["jkq"].reshape(sh + (nj,)), out["lstar"].reshape(sh),
            out["eb"].reshape(sh), out["b"].reshape((3,) + sh))


def jkq_vjp(prob, rho, g_jkq, g_lstar):
    """Gradients of sum(g_jkq J) + sum(g_lstar Lambda*) w.r.t. chi (fixed rho), rho, B."""
    nl = nl_of(prob.model)
    rho = _f64(rho).ravel(); gj = _f64(g_jkq).ravel(); gl = _f64(g_lstar).ravel()
    g_chi = np.zeros(prob.nvox); g_rho = np.zeros(prob.nvox * nl); g_b = np.zeros(3 * prob.nvox)
    rc = lib().or_jkq_vjp(prob.ref, _ptr(rho), _ptr(gj), _ptr(gl), _ptr(g_chi), _ptr(g_rho), _ptr(g_b))
    assert rc == 0, rc
    return g_chi.reshape(prob.shape), g_rho.reshape(prob.shape + (nl,)), g_b.reshape((3,) + prob.shape)


def emergent_vjp_rho(prob, rho, mu, chi, gout):
    """Adjoint of emergent in the unknowns: dL/dchi (fixed rho), dL/drho, dL/dB."""
    nl = nl_of(prob.model)
    rho = _f64(rho).ravel(); mu = _f64(mu); chi = _f64(chi); gout = _f64(gout).ravel()
    g_chi = np.zeros(prob.nvox); g_rho = np.zeros(prob.nvox * nl); g_b = np.zeros(3 * prob.nvox)
    rc = lib().or_emergent_vjp_rho(prob.ref, _ptr(rho), len(mu), _ptr(mu), _ptr(chi), _ptr(gout),
                                   _ptr(g_chi), _ptr(g_rho), _ptr(g_b))
    assert rc == 0, rc
    return g_chi.reshape(prob.shape), g_rho.reshape(prob.shape + (nl,)), g_b.reshape((3,) + prob.shape)


def initial_rho(prob, atm):
    """Starting point of the iteration: S^0_0 = B, all other components 0."""
    nl = nl_of(prob.model)
    rho = np.zeros(prob.shape + (nl,))
    rho[..., 0] = np.asarray(atm["bpl"]).reshape(prob.shape)
    return rho


def jacobi(prob, atm, rho=None, tol=1e-8, max_iter=1000):
    """Jacobi (ALI) iteration to a maximum relative change below tol."""
    rho = initial_rho(prob, atm) if rho is None else rho
    hist = []
    for _ in range(max_iter):
        jkq, ls = formal_solve(prob, rho)
        rho, mc = see_update(prob, jkq, ls, rho)
        hist.append(mc)
        if mc < tol:
            break
    return rho, hist


def flops_per_update(prob, rho, m=0, j=None):
    """Floating-point operations the oracle counts for one voxel.ray.frequency update
    (node coefficients counted once per node, not per interpolation corner)."""
    L = lib()
    j = prob.n_nu // 2 if j is None else j
    L.or_flops_reset(1)
    formal_solve(prob, rho, rays_range=(m, m + 1), freq_range=(j, j + 1))
    n = L.or_flops_get()
    L.or_flops_reset(0)
    return n / prob.nvox


def branch_signature(fn, *args, **kw):
    """Run fn(*args, **kw) with the control-point branch recorder on; returns
    (fn's result, signature). The signature hashes the sequence of BESSER branches
    (Sec. 3.2, steps 2, 6, 7, the parabola, and the linear last step) of every
    control point the oracle evaluated, in order: equal signatures mean the same
    branch was taken at every control point."""
    L = lib()
    L.or_branch_sig_reset(1)
    try:
        out = fn(*args, **kw)
        sig = int(L.or_branch_sig_get())
    finally:
        L.or_branch_sig_reset(0)
    return out, sig
