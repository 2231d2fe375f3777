"""torch.autograd.Function around the emergent Stokes profiles (forward:
porta_emergent_stokes; backward: porta_emergent_vjp, the hand-written adjoint
sweep). Argument marshalling only: both passes run in the CUDA library.

The differentiable inputs are per-voxel tensors on the context's device
(float64, shape (nz, ny, nx)): chi (line-centre opacity), e = chi S^0_0
(emission scale) and B (3, nz, ny, nx). The multipoles given to the solver
are ratios * e/chi, where ``ratios`` = rho^K_Q / S^0_0 (nz, ny, nx, nl) stays
fixed, as the gradient of porta_emergent_vjp assumes.
"""
import numpy as np
import torch


class EmergentStokes(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, fixed, mu, az, chi, e, B):
        """solver: binding.Context; fixed: dict of CUDA tensors vel, bpl, eps
        (per voxel) and ratios (per voxel and multipole); mu, az: host arrays
        of the outgoing directions. Returns [dir][nu][y][x][stokes]."""
        _load(solver, fixed, chi, e, B)
        nz, ny, nx = solver.shape
        out = torch.empty((len(mu), solver.nnu, ny, nx, solver.ns), dtype=torch.float64, device=chi.device)
        solver.emergent_stokes(mu, az, out)
        ctx.solver, ctx.fixed, ctx.mu, ctx.az = solver, fixed, mu, az
        ctx.save_for_backward(chi, e, B)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        chi, e, B = ctx.saved_tensors
        _load(ctx.solver, ctx.fixed, chi, e, B)      # the context may have been changed since forward
        g_chi, g_e, g_b = ctx.solver.emergent_vjp(ctx.mu, ctx.az, grad_out.contiguous())
        return None, None, None, None, g_chi, g_e, (g_b if B is not None else None)


def _load(solver, fixed, chi, e, B):
    atm = {"chi": chi.contiguous(), "eps": fixed["eps"], "bpl": fixed["bpl"], "vel": fixed["vel"]}
    if B is not None:
        atm.update(bx=B[0].contiguous(), by=B[1].contiguous(), bz=B[2].contiguous())
    solver.set_atmosphere(atm)
    solver.set_rho((fixed["ratios"] * (e / chi).unsqueeze(-1)).contiguous())


def emergent_stokes(solver, fixed, mu, az, chi, e, B=None):
    """Differentiable emergent Stokes profiles (see EmergentStokes)."""
    return EmergentStokes.apply(solver, fixed, np.asarray(mu, dtype=np.float64), np.asarray(az, dtype=np.float64),
                                chi, e, B)
