"""Gradients of an emergent-Stokes loss through Jacobi iterations (test
infrastructure only).

The unknowns start from S^0_0 = B (Planck), S^2_Q = 0 and take `niter`
Jacobi (ALI) iterations of the statistical-equilibrium equations (Sec. 2,
Eq. 2; the smoothing iteration of Sec. 5.1 without the coarse-grid correction), each a
formal solution (J^K_Q, Lambda-bar*) and an update; the loss is a function of
the emergent Stokes vector of the final unknowns. Parameters per voxel: the
line-centre opacity chi, the thermal emission term f = eps B of the
statistical equilibrium (its right-hand side, A(S) = f), and the field B.

Reverse mode with checkpoints: the forward pass keeps the unknowns every
`ckpt` iterations; the reverse pass recomputes the unknowns of each iteration
from the nearest checkpoint below it, then applies the reverse mode of the
update (or_see_update_vjp) and of the formal solution's J^K_Q and
Lambda-bar* (or_jkq_vjp).
"""
import numpy as np

from . import (Problem, emergent, emergent_vjp_rho, formal_solve, initial_rho, jkq_vjp, nl_of,
               see_update_src, see_update_vjp)


def _src(prob, f):
    nl = nl_of(prob.model)
    src = np.zeros(prob.shape + (nl,))
    src[..., 0] = f
    return src


def iterate(prob, rho, f, n):
    for _ in range(n):
        jkq, ls = formal_solve(prob, rho)
        rho, _ = see_update_src(prob, jkq, ls, rho, _src(prob, f))
    return rho


def forward(atm, model, quad, f, niter, mu, az):
    """Final unknowns and emergent Stokes vector for thermal term f."""
    prob = Problem(atm, model, *quad)
    rho = iterate(prob, initial_rho(prob, atm), f, niter)
    return rho, emergent(prob, rho, mu, az)


def loss_and_grad(atm, model, quad, f, niter, ckpt, mu, az, target):
    """L = sum (emergent - target)^2 and its gradients (chi, f, B) through niter iterations."""
    prob = Problem(atm, model, *quad)
    rho = initial_rho(prob, atm)
    saved = {0: rho.copy()}
    for k in range(niter):
        jkq, ls = formal_solve(prob, rho)
        rho, _ = see_update_src(prob, jkq, ls, rho, _src(prob, f))
        if (k + 1) % ckpt == 0:
            saved[k + 1] = rho.copy()
    out = emergent(prob, rho, mu, az)
    L = float(np.sum((out - target) ** 2))
    g_chi, g_rho, g_b = emergent_vjp_rho(prob, rho, mu, az, 2.0 * (out - target))
    g_f = np.zeros(prob.shape)
    for k in range(niter - 1, -1, -1):
        base = ckpt * (k // ckpt)
        rk = iterate(prob, saved[base].copy(), f, k - base)
        jkq, ls = formal_solve(prob, rk)
        # the update with src: f enters as eps B does, so dL/df is the eps-B gradient
        gr_expl, gj, gl, gf, gb = see_update_vjp(prob, jkq, ls, rk, g_rho, _src(prob, f))
        g_f += gf
        g_b += gb
        gc2, gr2, gb2 = jkq_vjp(prob, rk, gj, gl)
        g_chi += gc2
        g_b += gb2
        g_rho = gr_expl + gr2
    return L, g_chi, g_f, g_b, rho
