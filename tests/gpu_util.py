"""Helpers shared by the GPU parity tests: run the CUDA library and the oracle
on the same seeded inputs."""
import numpy as np

import oracle
import paper_1307_4217_gb300 as P
import synth


def make_ctx(atm, model, n_mu, n_chi, n_nu, precision, cluster=0, nu_group=0, rho=None):
    ctx = P.Context(atm, model, n_mu, n_chi, n_nu, precision=precision, cluster=cluster, nu_group=nu_group)
    ctx.set_atmosphere(atm)
    if rho is None:
        rho = initial_rho(atm, model)
    ctx.set_rho(rho)
    return ctx


def initial_rho(atm, model, seed=None):
    shape = (atm["nz"], atm["ny"], atm["nx"])
    nl = 1 if model == 0 else 6
    rho = np.zeros(shape + (nl,))
    rho[..., 0] = atm["bpl"]
    if seed is not None and nl > 1:
        rng = np.random.default_rng(seed)
        rho[..., 0] *= rng.uniform(0.7, 1.3, shape)
        rho[..., 1:] = 0.03 * rho[..., :1] * rng.normal(size=shape + (nl - 1,))
    return rho


def polarized_case(nx=12, ny=10, nz=16, seed=3):
    return synth.random_box(nx, ny, nz, seed=seed)


def unpolarized_case(nx=16, ny=16, nz=32, modulation=0.2, seed=None):
    atm = synth.plane_parallel_box(nx, ny, nz, modulation=modulation)
    if seed is not None:
        rng = np.random.default_rng(seed)
        atm["vel"] = 0.7 * rng.normal(size=atm["chi"].shape)
        atm["chi"] = atm["chi"] * np.exp(0.2 * rng.normal(size=atm["chi"].shape))
    return atm


def oracle_fs(atm, model, n_mu, n_chi, n_nu, rho):
    p = oracle.Problem(atm, model, n_mu, n_chi, n_nu)
    return p, oracle.formal_solve(p, rho)


def rel_err(a, b, scale=None):
    scale = np.abs(b) if scale is None else scale
    return float(np.max(np.abs(a - b) / scale))


# ---------------------------------------------------------------- oracle on all host cores

def _oracle_part(args):
    atm, model, quad, rho, m0, m1 = args
    p = oracle.Problem(atm, model, *quad)
    return oracle.formal_solve(p, rho, rays_range=(m0, m1))


_POOL = None


def oracle_pool():
    """Process pool for oracle formal solutions (spawned workers: safe to create
    after the CUDA context of the test process exists)."""
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        import os
        oracle.build()
        _POOL = mp.get_context("spawn").Pool(max(1, os.cpu_count() or 1))
    return _POOL


def oracle_fs_parallel(atm, model, quad, rho, chunks=None):
    """The oracle's formal solution (J^K_Q, Lambda-bar*) with its rays split into
    contiguous ranges over the host's cores; the partial sums are added in ray order."""
    import os
    nray = 2 * quad[0] * quad[1]
    n = chunks or min(nray, 4 * (os.cpu_count() or 1))
    edges = np.linspace(0, nray, n + 1).astype(int)
    jobs = [(atm, model, quad, rho, int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]
    parts = oracle_pool().map(_oracle_part, jobs)
    j = sum(p[0] for p in parts)
    l = sum(p[1] for p in parts)
    return j, l


def oracle_jacobi_parallel(atm, model, quad, tol, max_iter, rho=None):
    """Jacobi iteration of the oracle (formal solutions on all cores, update in this
    process) until the maximum change is below tol; returns (rho, changes)."""
    p = oracle.Problem(atm, model, *quad)
    rho = oracle.initial_rho(p, atm) if rho is None else rho
    hist = []
    for _ in range(max_iter):
        j, l = oracle_fs_parallel(atm, model, quad, rho)
        rho, mc = oracle.see_update(p, j, l, rho)
        hist.append(mc)
        if mc < tol:
            break
    return rho, hist
