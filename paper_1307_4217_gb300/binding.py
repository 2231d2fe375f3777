"""ctypes binding of include/porta.h: the same entry points under the same
names, plus a small ``Context`` convenience wrapper. Argument marshalling only.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); the ``where`` argument of the C ABI is derived from the array type.
"""
import ctypes
import os

import numpy as np

from . import build as _build

PORTA_OK, PORTA_EINVAL, PORTA_ENOMEM, PORTA_ECUDA, PORTA_ESTATE, PORTA_EKERNEL = 0, -1, -2, -3, -4, -7
PORTA_ENOTCONV = -5
PORTA_ESCRATCH = -8
PORTA_NOALLOC_SCRATCH_BYTES = 32 << 20
PORTA_MODEL_TWOLEVEL_UNPOL, PORTA_MODEL_TWOLEVEL_HANLE = 0, 1
PORTA_FP64, PORTA_FP32 = 0, 1
PORTA_HOST, PORTA_DEVICE = 0, 1
PORTA_SC_BESSER, PORTA_SC_PARABOLIC, PORTA_SC_LINEAR, PORTA_SC_BEZIER_FB, PORTA_SC_CBEZIER = 0, 1, 2, 3, 4

_STATUS = {0: "PORTA_OK", -1: "PORTA_EINVAL", -2: "PORTA_ENOMEM", -3: "PORTA_ECUDA", -4: "PORTA_ESTATE",
           -5: "PORTA_ENOTCONV",
           -7: "PORTA_EKERNEL", -8: "PORTA_ESCRATCH"}


def library_path():
    return _build.LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("z", ctypes.c_void_p)]


class _Atom(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("zeta", ctypes.c_double), ("gbar", ctypes.c_double),
                ("bcrit", ctypes.c_double)]


class _Quad(ctypes.Structure):
    _fields_ = [("n_mu", ctypes.c_int), ("n_chi", ctypes.c_int), ("n_nu", ctypes.c_int),
                ("x_max", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cluster", ctypes.c_int), ("nu_group", ctypes.c_int)]


class _Atmos(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz")]


class _MlAtom(ctypes.Structure):
    _fields_ = [("nlevel", ctypes.c_int), ("nline", ctypes.c_int), ("J", ctypes.c_void_p), ("E", ctypes.c_void_p),
                ("upper", ctypes.c_void_p), ("lower", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("eps", ctypes.c_void_p), ("polarized", ctypes.c_int), ("zeta", ctypes.c_double)]


_P, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_SIGS = {
    "porta_create": (_I, [_P, _P, _P, _P, _P]),
    "porta_batch_create": (_I, [_I, _P, _P, _P, _P, _P]),
    "porta_destroy": (None, [_P]),
    "porta_last_error": (ctypes.c_char_p, [_P]),
    "porta_set_stream": (_I, [_P, _P]),
    "porta_sizes": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "porta_rays": (_I, [_P, _P, _P, _P]),
    "porta_set_atmosphere": (_I, [_P, _P, _I]),
    "porta_set_rho": (_I, [_P, _P, _I]),
    "porta_get_rho": (_I, [_P, _P, _I]),
    "porta_formal_solve": (_I, [_P]),
    "porta_accumulate_jkq": (_I, [_P, _P, _P, _I]),
    "porta_see_update": (_I, [_P, _P]),
    "porta_emergent_stokes": (_I, [_P, _I, _P, _P, _P, _I]),
    "porta_probe_ray": (_I, [_P, _I, _P, _P, _I]),
    "porta_launch_info": (_I, [_P, _P, _P, _P, _P]),
    "porta_autotune": (_I, [_P, _P, _P]),
    "porta_run_iterations": (_I, [_P, _I, _P]),
    "porta_iterate_to": (_I, [_P, ctypes.c_double, _I, _I, _P, _P]),
    "porta_set_device_limit": (_I, [ctypes.c_longlong]),
    "porta_fma_peak": (_I, [_I, ctypes.c_double, _P, _P]),
    "porta_set_freq_range": (_I, [_P, _I, _I]),
    "porta_residual": (_I, [_P, _P]),
    "porta_eval_step": (_I, [_I, _I, _P, _P]),
    "porta_sigmoid_error": (_I, [_I, _I, _P, _P, _P, _P]),
    "porta_set_interpolation": (_I, [_P, _I]),
    "porta_set_explicit_medium": (_I, [_P, _P, _P, _I]),
    "porta_partial_size": (_I, [_P, _P, _P]),
    "porta_get_partial": (_I, [_P, _P, _I]),
    "porta_set_partial": (_I, [_P, _P, _I]),
    "porta_device_bytes": (ctypes.c_longlong, []),
    "porta_eval_coefficients": (_I, [_I, _I, _P, _P]),
    "porta_formal_solve_noalloc": (_I, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "porta_emergent_vjp": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _I]),
    "porta_set_adjoint_launch": (_I, [_P, _I, _I]),
    "porta_adjoint_info": (_I, [_P, _P, _P, _P, _P]),
    "porta_adjoint_timing": (_I, [_P, _P, _P]),
    "porta_fill_info": (_I, [_P, _P, _P, _P]),
    "porta_set_fill": (_I, [_P, _I, _I, _D]),
    "porta_mg_setup": (_I, [_P, _I]),
    "porta_mg_levels": (_I, [_P, _P, _P]),
    "porta_mg_vcycle": (_I, [_P, _I, _I, _I, _P]),
    "porta_mg_set_prolongation": (_I, [_P, _I]),
    "porta_mg_nested": (_I, [_P, _I, _I, _I, _I, _P]),
    "porta_iterate_ckpt": (_I, [_P, _I, _I, _P]),
    "porta_iterate_vjp": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _I]),
    "porta_set_tape_limit": (_I, [_P, ctypes.c_longlong]),
    "porta_iterate_timing": (_I, [_P, _P]),
    "porta_ml_create": (_I, [_P, _P, _P, _P, _P]),
    "porta_ml_set_atmosphere": (_I, [_P, _P, _P, _P, _P, _P, _P, _I]),
    "porta_ml_unknowns": (_I, [_P, _P]),
    "porta_ml_set_solve": (_I, [_P, _I]),
    "porta_set_sc_faces": (_I, [_P, _I]),
    "porta_set_global_sweep": (_I, [_P, _I]),
    "porta_ml_emergent_stokes": (_I, [_P, _I, _I, _P, _P, _P, _I]),
    "porta_ml_set_unknowns": (_I, [_P, _P, _I]),
    "porta_ml_get_unknowns": (_I, [_P, _P, _I]),
    "porta_ml_set_pops": (_I, [_P, _P, _I]),
    "porta_ml_get_pops": (_I, [_P, _P, _I]),
    "porta_ml_formal_solve": (_I, [_P, _P, _P, _I]),
    "porta_ml_see_update": (_I, [_P, _P]),
    "porta_ml_iterate": (_I, [_P, _I, _P]),
}

_lib = None


def lib(build_if_missing=True):
    """Load libporta_gb300.so (building it in-tree if missing). Raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = library_path()
        if build_if_missing and (not os.path.exists(path)):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PortaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _raw_ptr(a, n, dtype):
    """(pointer, where) of a contiguous buffer of n elements of dtype: a numpy
    array (host) or a CUDA tensor (device)."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous or a.size != n:
            raise TypeError(f"host buffer must be a contiguous {np.dtype(dtype).name} array of {n} elements")
        return a.ctypes.data, PORTA_HOST
    if getattr(a, "is_cuda", False):
        import torch
        want = torch.int64 if dtype == np.int64 else torch.float64
        if a.dtype != want or not a.is_contiguous() or a.numel() != n:
            raise TypeError(f"device buffer must be a contiguous {want} CUDA tensor of {n} elements")
        return a.data_ptr(), PORTA_DEVICE
    raise TypeError("buffer must be a numpy array or a CUDA tensor")


def _ptr_where(a):
    """(pointer, where, keepalive) for a numpy array or a CUDA tensor."""
    if a is None:
        return None, PORTA_HOST, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            a = np.ascontiguousarray(a, dtype=np.float64)
        return a.ctypes.data, PORTA_HOST, a
    # torch tensor
    if getattr(a, "is_cuda", False):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("device arrays must be contiguous float64 CUDA tensors")
        return a.data_ptr(), PORTA_DEVICE, a
    if a.__class__.__module__.startswith("torch"):
        import torch
        if a.dtype == torch.float64 and a.is_contiguous():
            return a.data_ptr(), PORTA_HOST, a      # host tensor (e.g. pinned memory), no copy
        a = a.detach().contiguous().to(torch.float64).numpy()
        return _ptr_where(a)
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data, PORTA_HOST, a


# ---- thin wrappers with the C names -------------------------------------------------

def porta_create(grid, atom, quad, opts):
    h = ctypes.c_void_p()
    rc = lib().porta_create(ctypes.byref(grid), ctypes.byref(atom), ctypes.byref(quad),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return rc, h


def porta_batch_create(grids, atom, quad, opts):
    arr = (_Grid * len(grids))(*grids)
    h = ctypes.c_void_p()
    rc = lib().porta_batch_create(len(grids), arr, ctypes.byref(atom), ctypes.byref(quad),
                                  ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return rc, h


def porta_destroy(h):
    lib().porta_destroy(h)


def porta_last_error(h):
    return lib().porta_last_error(h).decode()


def porta_set_stream(h, stream):
    return lib().porta_set_stream(h, stream)


def porta_sizes(h):
    nray, nnu, nl, nj, ns = (ctypes.c_int() for _ in range(5))
    nvox = ctypes.c_longlong()
    rc = lib().porta_sizes(h, ctypes.byref(nray), ctypes.byref(nnu), ctypes.byref(nvox), ctypes.byref(nl),
                           ctypes.byref(nj), ctypes.byref(ns))
    return rc, dict(nray=nray.value, nnu=nnu.value, nvox=nvox.value, nl=nl.value, nj=nj.value, ns=ns.value)


def porta_rays(h, nray):
    mu, chi, w = np.zeros(nray), np.zeros(nray), np.zeros(nray)
    rc = lib().porta_rays(h, mu.ctypes.data, chi.ctypes.data, w.ctypes.data)
    return rc, (mu, chi, w)


def porta_set_atmosphere(h, atmos, where):
    return lib().porta_set_atmosphere(h, ctypes.byref(atmos), where)


def porta_set_rho(h, ptr, where):
    return lib().porta_set_rho(h, ptr, where)


def porta_get_rho(h, ptr, where):
    return lib().porta_get_rho(h, ptr, where)


def porta_formal_solve(h):
    return lib().porta_formal_solve(h)


def porta_accumulate_jkq(h, jkq_ptr, lstar_ptr, where):
    return lib().porta_accumulate_jkq(h, jkq_ptr, lstar_ptr, where)


def porta_see_update(h, out=None):
    if out is None:
        return lib().porta_see_update(h, None)
    return lib().porta_see_update(h, ctypes.byref(out))


def porta_emergent_stokes(h, ndir, mu_ptr, chi_ptr, out_ptr, where):
    return lib().porta_emergent_stokes(h, ndir, mu_ptr, chi_ptr, out_ptr, where)


def porta_probe_ray(h, m, out_ptr, lstar_ptr, where):
    return lib().porta_probe_ray(h, m, out_ptr, lstar_ptr, where)


def porta_autotune(h):
    cl, nu = ctypes.c_int(), ctypes.c_int()
    rc = lib().porta_autotune(h, ctypes.byref(cl), ctypes.byref(nu))
    return rc, dict(cluster=cl.value, nu_group=nu.value)


def porta_eval_coefficients(precision, t):
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.zeros((len(t), 6))
    rc = lib().porta_eval_coefficients(precision, len(t), t.ctypes.data, out.ctypes.data)
    return rc, out


def porta_formal_solve_noalloc(atm, model, n_mu, n_chi, n_nu, x_max, datm, rho_ptr, jkq_ptr, lstar_ptr, stream=None):
    """Allocation-free formal solution: descriptions from ``atm`` (host), device
    pointers for the atmosphere arrays (``datm``: dict of CUDA tensors), rho and the outputs."""
    z = np.ascontiguousarray(atm["z"], dtype=np.float64)
    g = _Grid(atm["nx"], atm["ny"], atm["nz"], float(atm["lx"]), float(atm["ly"]), z.ctypes.data)
    a = _Atom(model, float(atm.get("zeta", 0.0)), float(atm.get("gbar", 1.0)), float(atm.get("bcrit", 25.0)))
    q = _Quad(n_mu, n_chi, n_nu, float(x_max))
    ptrs = [datm[k].data_ptr() if datm.get(k) is not None else None
            for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz")]
    s = _Atmos(*ptrs)
    handle = getattr(stream, "cuda_stream", stream)
    return lib().porta_formal_solve_noalloc(ctypes.byref(g), ctypes.byref(a), ctypes.byref(q), ctypes.byref(s),
                                            rho_ptr, jkq_ptr, lstar_ptr, ctypes.c_void_p(handle or 0))


def porta_run_iterations(h, iterations, out=None):
    return lib().porta_run_iterations(h, iterations, ctypes.byref(out) if out is not None else None)


def porta_fma_peak(kind, seconds=1.0):
    """Measured FMA peak: kind 0 FP32, 1 packed FP32 (float2), 2 FP64. Returns (status, TFLOP/s, ms)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib().porta_fma_peak(int(kind), float(seconds), ctypes.byref(tf), ctypes.byref(ms))
    return rc, tf.value, ms.value


def porta_eval_step(precision, cases):
    """The GPU's general BESSER-DELO step on rows of 34 inputs; returns (status, [n][5] outputs)."""
    cases = np.ascontiguousarray(cases, dtype=np.float64).reshape(-1, 34)
    out = np.zeros((cases.shape[0], 5))
    rc = lib().porta_eval_step(int(precision), cases.shape[0], cases.ctypes.data, out.ctypes.data)
    return rc, out


def porta_sigmoid_error(precision, method, dtau, shift=None):
    """E(dtau) of the sigmoid benchmark (Sec. 3.4) for each case (method, dtau, shift),
    solved on the GPU; returns (status, E)."""
    dtau = np.ascontiguousarray(dtau, dtype=np.float64).ravel()
    method = np.ascontiguousarray(np.broadcast_to(method, dtau.shape), dtype=np.int32)
    shift = np.zeros_like(dtau) if shift is None else np.ascontiguousarray(np.broadcast_to(shift, dtau.shape),
                                                                            dtype=np.float64)
    E = np.zeros_like(dtau)
    rc = lib().porta_sigmoid_error(int(precision), dtau.size, method.ctypes.data, dtau.ctypes.data,
                                   shift.ctypes.data, E.ctypes.data)
    return rc, E


def porta_set_interpolation(h, order):
    return lib().porta_set_interpolation(h, int(order))


def porta_set_explicit_medium(h, kexpl_ptr, sexpl_ptr, where):
    return lib().porta_set_explicit_medium(h, kexpl_ptr, sexpl_ptr, where)


def porta_residual(h):
    r = ctypes.c_double()
    rc = lib().porta_residual(h, ctypes.byref(r))
    return rc, r.value


def porta_set_freq_range(h, j0, j1):
    return lib().porta_set_freq_range(h, int(j0), int(j1))


def porta_partial_size(h):
    n, b = ctypes.c_longlong(), ctypes.c_int()
    rc = lib().porta_partial_size(h, ctypes.byref(n), ctypes.byref(b))
    return rc, n.value, b.value


def porta_get_partial(h, out, where):
    return lib().porta_get_partial(h, out, where)


def porta_set_partial(h, buf, where):
    return lib().porta_set_partial(h, buf, where)


def porta_set_device_limit(nbytes):
    """Process-wide cap on the library's device allocations (0: none)."""
    return lib().porta_set_device_limit(int(nbytes))


def porta_device_bytes():
    return lib().porta_device_bytes()


def porta_iterate_to(h, tol, max_iter, check_every=1):
    """Returns (status, iterations done, last maximum change)."""
    n, ch = ctypes.c_int(), ctypes.c_double()
    rc = lib().porta_iterate_to(h, float(tol), int(max_iter), int(check_every), ctypes.byref(n), ctypes.byref(ch))
    return rc, n.value, ch.value


def porta_launch_info(h):
    v = [ctypes.c_int() for _ in range(4)]
    rc = lib().porta_launch_info(h, *[ctypes.byref(x) for x in v])
    return rc, dict(clusters=v[0].value, cluster=v[1].value, nu_group=v[2].value, smem=v[3].value)


def porta_emergent_vjp(h, ndir, mu_ptr, chi_ptr, grad_ptr, out_ptr, gchi_ptr, ge_ptr, gb_ptr, where):
    return lib().porta_emergent_vjp(h, ndir, mu_ptr, chi_ptr, grad_ptr, out_ptr, gchi_ptr, ge_ptr, gb_ptr, where)


def porta_set_adjoint_launch(h, cluster, nu_group):
    return lib().porta_set_adjoint_launch(h, cluster, nu_group)


def porta_adjoint_info(h):
    v = [ctypes.c_int() for _ in range(4)]
    rc = lib().porta_adjoint_info(h, *[ctypes.byref(x) for x in v])
    return rc, dict(clusters=v[0].value, cluster=v[1].value, nu_group=v[2].value, smem=v[3].value)


def porta_adjoint_timing(h):
    f, a = ctypes.c_float(), ctypes.c_float()
    rc = lib().porta_adjoint_timing(h, ctypes.byref(f), ctypes.byref(a))
    return rc, dict(forward_ms=f.value, adjoint_ms=a.value)


def porta_fill_info(h):
    cl, nu, fr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    rc = lib().porta_fill_info(h, ctypes.byref(cl), ctypes.byref(nu), ctypes.byref(fr))
    return rc, dict(cluster=cl.value, nu_group=nu.value, fraction=fr.value)


def porta_set_fill(h, cluster, nu_group, fraction):
    return lib().porta_set_fill(h, cluster, nu_group, float(fraction))


def porta_mg_setup(h, nlevels):
    return lib().porta_mg_setup(h, nlevels)


def porta_mg_levels(h):
    n = ctypes.c_int()
    shapes = (ctypes.c_int * 24)()
    rc = lib().porta_mg_levels(h, ctypes.byref(n), shapes)
    return rc, [tuple(shapes[3 * l:3 * l + 3]) for l in range(n.value)]


def porta_mg_vcycle(h, npre, npost, ncoarse, out=None):
    return lib().porta_mg_vcycle(h, npre, npost, ncoarse, ctypes.byref(out) if out is not None else None)


def porta_mg_set_prolongation(h, order):
    return lib().porta_mg_set_prolongation(h, int(order))


def porta_mg_nested(h, ncycles, npre, npost, ncoarse, out=None):
    return lib().porta_mg_nested(h, ncycles, npre, npost, ncoarse, ctypes.byref(out) if out is not None else None)


def porta_iterate_ckpt(h, niter, ckpt, out=None):
    return lib().porta_iterate_ckpt(h, niter, ckpt, ctypes.byref(out) if out is not None else None)


def porta_iterate_vjp(h, ndir, mu_ptr, chi_ptr, grad_ptr, out_ptr, gchi_ptr, gf_ptr, gb_ptr, where):
    return lib().porta_iterate_vjp(h, ndir, mu_ptr, chi_ptr, grad_ptr, out_ptr, gchi_ptr, gf_ptr, gb_ptr, where)


def porta_set_tape_limit(h, nbytes):
    return lib().porta_set_tape_limit(h, int(nbytes))


def porta_iterate_timing(h):
    ms = (ctypes.c_float * 5)()
    rc = lib().porta_iterate_timing(h, ms)
    keys = ("recompute_ms", "see_adjoint_ms", "tape_forward_ms", "jkq_adjoint_ms", "reduce_ms")
    return rc, dict(zip(keys, list(ms)))


def porta_ml_create(grid, atom, quad, opts):
    h = ctypes.c_void_p()
    rc = lib().porta_ml_create(ctypes.byref(grid), ctypes.byref(atom), ctypes.byref(quad),
                               ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return rc, h


def porta_ml_set_atmosphere(h, chi_ptr, kt_ptr, vel_ptr, bx_ptr, by_ptr, bz_ptr, where):
    return lib().porta_ml_set_atmosphere(h, chi_ptr, kt_ptr, vel_ptr, bx_ptr, by_ptr, bz_ptr, where)


def porta_ml_emergent_stokes(h, line, ndir, mu_ptr, chi_ptr, out_ptr, where):
    return lib().porta_ml_emergent_stokes(h, line, ndir, mu_ptr, chi_ptr, out_ptr, where)


def porta_set_sc_faces(h, on):
    return lib().porta_set_sc_faces(h, on)


def porta_set_global_sweep(h, on):
    return lib().porta_set_global_sweep(h, on)


def porta_ml_set_solve(h, mode):
    return lib().porta_ml_set_solve(h, mode)


def porta_ml_unknowns(h):
    n = ctypes.c_int()
    rc = lib().porta_ml_unknowns(h, ctypes.byref(n))
    return rc, n.value


def porta_ml_set_unknowns(h, ptr, where):
    return lib().porta_ml_set_unknowns(h, ptr, where)


def porta_ml_get_unknowns(h, ptr, where):
    return lib().porta_ml_get_unknowns(h, ptr, where)


def porta_ml_set_pops(h, ptr, where):
    return lib().porta_ml_set_pops(h, ptr, where)


def porta_ml_get_pops(h, ptr, where):
    return lib().porta_ml_get_pops(h, ptr, where)


def porta_ml_formal_solve(h, jbar_ptr, lstar_ptr, where):
    return lib().porta_ml_formal_solve(h, jbar_ptr, lstar_ptr, where)


def porta_ml_see_update(h, out=None):
    return lib().porta_ml_see_update(h, ctypes.byref(out) if out is not None else None)


def porta_ml_iterate(h, iterations, out=None):
    return lib().porta_ml_iterate(h, iterations, ctypes.byref(out) if out is not None else None)


# ---- convenience wrapper ------------------------------------------------------------

class Context:
    """One solver context (grid + atom + quadratures) on the current CUDA device.

    ``atm`` is a dict with nx, ny, nz, lx, ly, z and the atomic constants zeta,
    gbar, bcrit (as produced by ``synth``).
    """

    def __init__(self, atm, model, n_mu, n_chi, n_nu, x_max=4.0, precision=PORTA_FP32, cluster=0, nu_group=0):
        self._keep = []
        z = np.ascontiguousarray(atm["z"], dtype=np.float64)
        self._keep.append(z)
        g = _Grid(atm["nx"], atm["ny"], atm["nz"], float(atm["lx"]), float(atm["ly"]), z.ctypes.data)
        a = _Atom(model, float(atm.get("zeta", 0.0)), float(atm.get("gbar", 1.0)), float(atm.get("bcrit", 25.0)))
        q = _Quad(n_mu, n_chi, n_nu, float(x_max))
        o = _Opts(precision, cluster, nu_group)
        self.h = None
        rc, h = porta_create(g, a, q, o)
        if rc != PORTA_OK:
            raise PortaError(rc, "porta_create failed")
        self.h = h
        rc, s = porta_sizes(h)
        self.__dict__.update(s)
        self.shape = (atm["nz"], atm["ny"], atm["nx"])
        self.model = model
        self.precision = precision

    def close(self):
        if self.h is not None:
            porta_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != PORTA_OK:
            raise PortaError(rc, porta_last_error(self.h))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer handle, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(porta_set_stream(self.h, ctypes.c_void_p(handle or 0)))

    def rays(self):
        rc, r = porta_rays(self.h, self.nray)
        self._check(rc)
        return r

    def set_atmosphere(self, atm):
        arrs = {}
        where = None
        for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz"):
            v = atm.get(k)
            if v is None:
                arrs[k] = None
                continue
            p, w, keep = _ptr_where(v)
            arrs[k] = p
            self._keep.append(keep)
            where = w if where is None else where
            if w != where:
                raise TypeError("atmosphere arrays must all be host or all device")
        s = _Atmos(*[arrs[k] for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz")])
        self._check(porta_set_atmosphere(self.h, s, where))

    def set_rho(self, rho):
        p, w, keep = _ptr_where(rho)
        self._check(porta_set_rho(self.h, p, w))

    def get_rho(self, out=None):
        if out is None:
            out = np.zeros(self.shape + (self.nl,))
        p, w, keep = _ptr_where(out)
        self._check(porta_get_rho(self.h, p, w))
        return out if w == PORTA_DEVICE or keep is out else keep.reshape(self.shape + (self.nl,))

    def formal_solve(self):
        self._check(porta_formal_solve(self.h))

    def accumulate_jkq(self, jkq=None, lstar=None, want=True):
        if want and jkq is None:
            jkq = np.zeros(self.shape + (self.nj,))
            lstar = np.zeros(self.shape)
        pj, wj, kj = _ptr_where(jkq)
        pl, wl, kl = _ptr_where(lstar)
        where = wj if jkq is not None else wl
        self._check(porta_accumulate_jkq(self.h, pj, pl, where))
        return jkq, lstar

    def residual(self):
        """max relative residual of A(x) = f at the current unknowns (porta_residual)."""
        rc, r = porta_residual(self.h)
        self._check(rc)
        return r

    # ---- frequency bands (multi-GPU splitting of a formal solution)
    def set_freq_range(self, j0, j1):
        """Sweep only the frequencies [j0, j1) in later formal solutions ((0, 0): all)."""
        self._check(porta_set_freq_range(self.h, j0, j1))

    def partial_dtype(self):
        """numpy dtype of the partial sums: int64 fixed point (FP32 form) or float64."""
        return np.int64 if self.precision == PORTA_FP32 else np.float64

    def get_partial(self, out=None):
        """The last formal solution's partial sums of J^K_Q and Lambda-bar* into `out`
        (a numpy array or a contiguous CUDA tensor of partial_dtype(), partial_size()
        elements); a new numpy array if out is None."""
        rc, n, _ = porta_partial_size(self.h)
        self._check(rc)
        if out is None:
            out = np.zeros(n, dtype=self.partial_dtype())
        ptr, where = _raw_ptr(out, n, self.partial_dtype())
        self._check(porta_get_partial(self.h, ptr, where))
        return out

    def set_partial(self, buf):
        """Make summed partial sums (same layout as get_partial) this context's J^K_Q and
        Lambda-bar* for the next see_update."""
        rc, n, _ = porta_partial_size(self.h)
        self._check(rc)
        ptr, where = _raw_ptr(buf, n, self.partial_dtype())
        self._check(porta_set_partial(self.h, ptr, where))

    def see_update(self, residual=True):
        if not residual:
            self._check(porta_see_update(self.h, None))
            return None
        out = ctypes.c_double()
        self._check(porta_see_update(self.h, out))
        return out.value

    def emergent_stokes(self, mu, chi, out=None):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        nz, ny, nx = self.shape
        if out is None:
            out = np.zeros((len(mu), self.nnu, ny, nx, self.ns))
        p, w, keep = _ptr_where(out)
        self._check(porta_emergent_stokes(self.h, len(mu), mu.ctypes.data, chi.ctypes.data, p, w))
        return out

    def emergent_vjp(self, mu, chi, grad_out, out=None, g_chi=None, g_e=None, g_b=None):
        """Gradients of sum(grad_out * emergent_stokes(mu, chi)) with respect to per-voxel chi,
        e = chi S^0_0 (multipole ratios fixed) and B: returns (g_chi, g_e, g_b[, out]).
        grad_out and the optional output arrays are all numpy (host) or all CUDA tensors."""
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        pg, where, kg = _ptr_where(grad_out)
        if g_chi is None:
            if where == PORTA_DEVICE:
                import torch
                dev = grad_out.device
                g_chi = torch.empty(self.shape, dtype=torch.float64, device=dev)
                g_e = torch.empty(self.shape, dtype=torch.float64, device=dev)
                g_b = torch.empty((3,) + self.shape, dtype=torch.float64, device=dev)
            else:
                g_chi, g_e, g_b = np.zeros(self.shape), np.zeros(self.shape), np.zeros((3,) + self.shape)
        ptrs = []
        for arr in (out, g_chi, g_e, g_b):
            p, w, keep = _ptr_where(arr)
            if arr is not None and w != where:
                raise TypeError("grad_out and the outputs must all be host or all device")
            ptrs.append(p)
        self._check(porta_emergent_vjp(self.h, len(mu), mu.ctypes.data, chi.ctypes.data, pg, *ptrs, where))
        return (g_chi, g_e, g_b) if out is None else (g_chi, g_e, g_b, out)

    def iterate_ckpt(self, niter, ckpt, residual=True):
        """niter Jacobi iterations from the current rho keeping a checkpoint of rho
        every ckpt iterations (for iterate_vjp); returns the last update's change."""
        out = ctypes.c_double() if residual else None
        self._check(porta_iterate_ckpt(self.h, niter, ckpt, out))
        return out.value if residual else None

    def iterate_vjp(self, mu, chi, grad_out, out=None, g_chi=None, g_f=None, g_b=None):
        """Gradients of sum(grad_out * emergent_stokes(mu, chi)) at the last iterate of
        iterate_ckpt with respect to per-voxel chi, the thermal term f = eps B and B,
        through the iterations: returns (g_chi, g_f, g_b[, out]). grad_out and the
        optional output arrays are all numpy (host) or all CUDA tensors."""
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        pg, where, kg = _ptr_where(grad_out)
        if g_chi is None:
            if where == PORTA_DEVICE:
                import torch
                dev = grad_out.device
                g_chi = torch.empty(self.shape, dtype=torch.float64, device=dev)
                g_f = torch.empty(self.shape, dtype=torch.float64, device=dev)
                g_b = torch.empty((3,) + self.shape, dtype=torch.float64, device=dev)
            else:
                g_chi, g_f, g_b = np.zeros(self.shape), np.zeros(self.shape), np.zeros((3,) + self.shape)
        ptrs = []
        for arr in (out, g_chi, g_f, g_b):
            p, w, keep = _ptr_where(arr)
            if arr is not None and w != where:
                raise TypeError("grad_out and the outputs must all be host or all device")
            ptrs.append(p)
        self._check(porta_iterate_vjp(self.h, len(mu), mu.ctypes.data, chi.ctypes.data, pg, *ptrs, where))
        return (g_chi, g_f, g_b) if out is None else (g_chi, g_f, g_b, out)

    def iterate_timing(self):
        rc, t = porta_iterate_timing(self.h)
        self._check(rc)
        return t

    def set_tape_limit(self, nbytes=0):
        """Device bytes for the per-batch forward tape of iterate_vjp (0: 16 GB)."""
        self._check(porta_set_tape_limit(self.h, nbytes))

    def set_adjoint_launch(self, cluster=0, nu_group=0):
        self._check(porta_set_adjoint_launch(self.h, cluster, nu_group))

    def adjoint_info(self):
        rc, info = porta_adjoint_info(self.h)
        self._check(rc)
        return info

    def adjoint_timing(self):
        rc, t = porta_adjoint_timing(self.h)
        self._check(rc)
        return t

    def probe_ray(self, m):
        out = np.zeros((self.nnu,) + self.shape + (self.ns,))
        ls = np.zeros((self.nnu,) + self.shape)
        self._check(porta_probe_ray(self.h, m, out.ctypes.data, ls.ctypes.data, PORTA_HOST))
        return out, ls

    def run_iterations(self, n, residual=True):
        """n Jacobi iterations replayed from a captured CUDA graph (needs set_stream)."""
        out = ctypes.c_double() if residual else None
        self._check(porta_run_iterations(self.h, n, out))
        return out.value if residual else None

    def iterate_to(self, tol, max_iter, check_every=1):
        """Jacobi iterations (graph replay) until the maximum change is below tol.
        Returns (iterations, last change, converged); PORTA_ENOTCONV is reported as
        converged = False, every other error raises."""
        rc, n, ch = porta_iterate_to(self.h, tol, max_iter, check_every)
        if rc == PORTA_ENOTCONV:
            return n, ch, False
        self._check(rc)
        return n, ch, True

    def autotune(self):
        rc, r = porta_autotune(self.h)
        self._check(rc)
        return r

    def launch_info(self):
        rc, info = porta_launch_info(self.h)
        self._check(rc)
        return info

    def mg_setup(self, nlevels):
        self._check(porta_mg_setup(self.h, nlevels))

    def mg_levels(self):
        rc, shapes = porta_mg_levels(self.h)
        self._check(rc)
        return shapes

    def mg_vcycle(self, npre=2, npost=4, ncoarse=8, residual=True):
        """One multigrid V-cycle; returns the maximum relative change of rho (or None)."""
        out = ctypes.c_double() if residual else None
        self._check(porta_mg_vcycle(self.h, npre, npost, ncoarse, out))
        return out.value if residual else None

    def set_explicit_medium(self, kexpl=None, sexpl=None):
        """Explicit medium for the emergent profiles: kexpl (6, nz, ny, nx) =
        (eta_Q, eta_U, eta_V, rho_Q, rho_U, rho_V) / eta_I and sexpl (4, nz, ny, nx) = S
        (host arrays); None clears it."""
        if kexpl is None or sexpl is None:
            self._check(porta_set_explicit_medium(self.h, None, None, PORTA_HOST))
            return
        k = np.ascontiguousarray(kexpl, dtype=np.float64)
        s = np.ascontiguousarray(sexpl, dtype=np.float64)
        self._check(porta_set_explicit_medium(self.h, k.ctypes.data, s.ctypes.data, PORTA_HOST))

    def set_interpolation(self, order):
        """Interpolation at M and P: 1 bilinear, 2 biquadratic (Sec. 3.1)."""
        self._check(porta_set_interpolation(self.h, order))

    def set_sc_faces(self, on):
        """1: short characteristics end on the first cell face they cross (vertical
        faces included, Sec. 3.1); 0: on the next horizontal plane."""
        self._check(porta_set_sc_faces(self.h, int(on)))

    def set_global_sweep(self, on):
        """1: the J^K_Q formal solution by the global-memory sweep in the plane
        placement (taken by itself where no shared-memory sweep fits); 0: the
        shared-memory sweeps where they fit."""
        self._check(porta_set_global_sweep(self.h, int(on)))

    def mg_set_prolongation(self, order):
        """Prolongation of the multigrid cycles: 1 tri-linear, 3 tri-cubic-centered."""
        self._check(porta_mg_set_prolongation(self.h, order))

    def mg_nested(self, ncycles=1, npre=2, npost=4, ncoarse=8, residual=True):
        """Nested multigrid from the coarsest grid up; returns the maximum relative change
        over the finest level's last V-cycle (or None)."""
        out = ctypes.c_double() if residual else None
        self._check(porta_mg_nested(self.h, ncycles, npre, npost, ncoarse, out))
        return out.value if residual else None

    def set_fill(self, cluster=0, nu_group=0, fraction=0.0):
        self._check(porta_set_fill(self.h, cluster, nu_group, fraction))

    def fill_info(self):
        rc, info = porta_fill_info(self.h)
        self._check(rc)
        return info


class BatchContext(Context):
    """Several independent boxes of uneven size sharing atom and quadratures
    (porta_batch_create). Voxel arrays are the boxes' arrays (raveled in
    (nz, ny, nx) order) concatenated in box order; results come back the same way."""

    def __init__(self, atms, model, n_mu, n_chi, n_nu, x_max=4.0, precision=PORTA_FP32, cluster=0, nu_group=0):
        self._keep = []
        grids = []
        for atm in atms:
            z = np.ascontiguousarray(atm["z"], dtype=np.float64)
            self._keep.append(z)
            grids.append(_Grid(atm["nx"], atm["ny"], atm["nz"], float(atm["lx"]), float(atm["ly"]), z.ctypes.data))
        a0 = atms[0]
        a = _Atom(model, float(a0.get("zeta", 0.0)), float(a0.get("gbar", 1.0)), float(a0.get("bcrit", 25.0)))
        q = _Quad(n_mu, n_chi, n_nu, float(x_max))
        o = _Opts(precision, cluster, nu_group)
        self.h = None
        rc, h = porta_batch_create(grids, a, q, o)
        if rc != PORTA_OK:
            raise PortaError(rc, "porta_batch_create failed")
        self.h = h
        rc, s = porta_sizes(h)
        self.__dict__.update(s)
        self.box_sizes = [int(t["nx"]) * int(t["ny"]) * int(t["nz"]) for t in atms]
        self.offsets = np.concatenate([[0], np.cumsum(self.box_sizes)])
        self.shape = (int(self.offsets[-1]),)
        self.model = model
        self.precision = precision

    @staticmethod
    def concat(atms, key):
        if atms[0].get(key) is None:
            return None
        return np.concatenate([np.asarray(t[key], dtype=np.float64).ravel() for t in atms])

    def set_atmosphere(self, atms):
        Context.set_atmosphere(self, {k: self.concat(atms, k) for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz")})

    def split(self, arr):
        """Per-box views of a concatenated voxel array."""
        return [arr[self.offsets[b]:self.offsets[b + 1]] for b in range(len(self.box_sizes))]


class MlContext(Context):
    """Multilevel atom without polarization (porta_ml_create): ``atom`` as
    produced by ``synth.multilevel_atom`` (J, E, lines (upper, lower), A, eps),
    ``atm`` with nx, ny, nz, lx, ly, z. Line arrays come back [line][voxel]."""

    def __init__(self, atm, atom, n_mu, n_chi, n_nu, x_max=4.0, precision=PORTA_FP32, cluster=0, nu_group=0,
                 polarized=False, zeta=None):
        self._keep = []
        z = np.ascontiguousarray(atm["z"], dtype=np.float64)
        J = np.ascontiguousarray(atom["J"], dtype=np.float64)
        E = np.ascontiguousarray(atom["E"], dtype=np.float64)
        lines = np.asarray(atom["lines"])
        up = np.ascontiguousarray(lines[:, 0], dtype=np.int32)
        lo = np.ascontiguousarray(lines[:, 1], dtype=np.int32)
        A = np.ascontiguousarray(atom["A"], dtype=np.float64)
        eps = np.ascontiguousarray(atom["eps"], dtype=np.float64)
        self._keep += [z, J, E, up, lo, A, eps]
        g = _Grid(atm["nx"], atm["ny"], atm["nz"], float(atm["lx"]), float(atm["ly"]), z.ctypes.data)
        if zeta is None:
            zeta = float(atm.get("zeta", 0.0))
        a = _MlAtom(len(J), len(A), J.ctypes.data, E.ctypes.data, up.ctypes.data, lo.ctypes.data, A.ctypes.data,
                    eps.ctypes.data, 1 if polarized else 0, float(zeta))
        q = _Quad(n_mu, n_chi, n_nu, float(x_max))
        o = _Opts(precision, cluster, nu_group)
        self.h = None
        rc, h = porta_ml_create(g, a, q, o)
        if rc != PORTA_OK:
            raise PortaError(rc, "porta_ml_create failed")
        self.h = h
        rc, s = porta_sizes(h)
        self.__dict__.update(s)
        self.grid_shape = (atm["nz"], atm["ny"], atm["nx"])
        self.nlevel, self.nline = len(J), len(A)
        self.polarized = bool(polarized)
        self.shape = (self.nline,) + self.grid_shape
        self.model = None
        rc, self.nunk = porta_ml_unknowns(h)
        self._check(rc)

    def set_atmosphere(self, atm):
        ptrs, where = [], None
        for k in ("chi", "kT", "vel", "bx", "by", "bz"):
            if atm.get(k) is None:
                ptrs.append(None)
                continue
            v = atm[k] if hasattr(atm[k], "data_ptr") else np.asarray(atm[k], dtype=np.float64)
            p, w, keep = _ptr_where(v)
            self._keep.append(keep)
            where = w if where is None else where
            if w != where:
                raise TypeError("atmosphere arrays must all be host or all device")
            ptrs.append(p)
        self._check(porta_ml_set_atmosphere(self.h, *ptrs, where))

    def emergent_stokes(self, line, mu, chi, out=None):
        """emergent Stokes profiles of line `line` along (mu, chi): [dir][nu][y][x][stokes]"""
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        nz, ny, nx = self.grid_shape
        if out is None:
            out = np.zeros((len(mu), self.nnu, ny, nx, self.ns))
        p, w, keep = _ptr_where(out)
        self._check(porta_ml_emergent_stokes(self.h, line, len(mu), mu.ctypes.data, chi.ctypes.data, p, w))
        return out

    def set_solve(self, mode):
        """rate equations of the polarized atom: 0 FP32 factors with FP64 refinement
        (default), 1 FP64 elimination"""
        self._check(porta_ml_set_solve(self.h, mode))

    def set_unknowns(self, x):
        """the vector of unknowns [voxel][nunk] (populations, or the real multipoles
        level, K, rho^K_0, Re/Im rho^K_Q (Q = 1..K) of the polarized atom)"""
        if not hasattr(x, "data_ptr"):
            x = np.ascontiguousarray(x, dtype=np.float64)
        p, w, keep = _ptr_where(x)
        self._check(porta_ml_set_unknowns(self.h, p, w))

    def get_unknowns(self, out=None):
        if out is None:
            out = np.zeros(self.grid_shape + (self.nunk,))
        p, w, keep = _ptr_where(out)
        self._check(porta_ml_get_unknowns(self.h, p, w))
        return out

    def set_pops(self, pops):
        if not hasattr(pops, "data_ptr"):
            pops = np.ascontiguousarray(pops, dtype=np.float64)
        p, w, keep = _ptr_where(pops)
        self._check(porta_ml_set_pops(self.h, p, w))

    def get_pops(self, out=None):
        if out is None:
            out = np.zeros(self.grid_shape + (self.nlevel,))
        p, w, keep = _ptr_where(out)
        self._check(porta_ml_get_pops(self.h, p, w))
        return out

    def ml_formal_solve(self, jbar=None, lstar=None, want=True):
        """Formal solution of every line; returns (Jbar, Lambda-bar*) [line][voxel] or (None, None).
        Polarized atom: Jbar [line][voxel][9] = (J00, J10, Re J11, Im J11, J20, Re J21, Im J21,
        Re J22, Im J22)."""
        if want and jbar is None:
            jbar = np.zeros(self.shape + ((9,) if self.polarized else ()))
            lstar = np.zeros(self.shape)
        pj, wj, kj = _ptr_where(jbar)
        pl, wl, kl = _ptr_where(lstar)
        where = wj if jbar is not None else (wl if lstar is not None else PORTA_DEVICE)
        self._check(porta_ml_formal_solve(self.h, pj, pl, where))
        return jbar, lstar

    def ml_see_update(self, residual=True):
        out = ctypes.c_double() if residual else None
        self._check(porta_ml_see_update(self.h, out))
        return out.value if residual else None

    def ml_iterate(self, n, residual=True):
        out = ctypes.c_double() if residual else None
        self._check(porta_ml_iterate(self.h, n, out))
        return out.value if residual else None
