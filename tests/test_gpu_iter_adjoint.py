"""Gradients through Jacobi iterations on the GPU (porta_iterate_ckpt /
porta_iterate_vjp) against the oracle's checkpointed FP64 reverse mode
(oracle/diff.py, itself pinned to central differences of the forward
iterations).

Tolerances. FP64: the two sides differentiate the same iterations in a
different order and form, so the gradients agree to rounding amplified by
the sums over rays, frequencies and iterations: 1e-8 of the largest
component. FP32: the sweeps carry 1e-5 relative error into J^K_Q, every
step back multiplies gradients by a few such factors, and the thick-layer
cancellation of the Zeeman terms in the B gradient amplifies them (as for
the single-formal-solution adjoint): 2e-3 of the largest component and 2e-3
in the relative 2-norm.
"""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import make_ctx
from oracle import diff

pytestmark = pytest.mark.gpu

QUAD = (2, 4, 3)


def _case(pol, nx=6, ny=5, nz=9, seed=3):
    if pol:
        atm = synth.random_box(nx, ny, nz, seed=seed, tau_top=1e-2, tau_bot=1e2)
        for k in ("bx", "by", "bz"):
            atm[k] = atm[k] * 50.0
    else:
        atm = synth.plane_parallel_box(nx, ny, nz, modulation=0.3, tau_top=1e-2, tau_bot=1e2)
        atm["vel"] = 0.5 * np.random.default_rng(seed).normal(size=atm["chi"].shape)
    atm["eps"] = np.full_like(atm["eps"], 0.05)
    # a varying Planck function keeps the first iterates off BESSER's kinks
    atm["bpl"] = np.exp(0.3 * np.random.default_rng(seed + 8).normal(size=atm["chi"].shape))
    return atm, (1 if pol else 0)


def _oracle(atm, model, niter, ckpt, mu, az, gout):
    """Oracle gradients of sum(gout * emergent) through niter iterations: the
    quadratic loss with target = out - gout / 2 has dL/dout = gout."""
    f = np.asarray(atm["eps"]) * np.asarray(atm["bpl"])
    rho, out = diff.forward(atm, model, QUAD, f, niter, mu, az)
    _, g_chi, g_f, g_b, rho2 = diff.loss_and_grad(atm, model, QUAD, f, niter, ckpt, mu, az, out - 0.5 * gout)
    assert np.array_equal(rho, rho2)
    return rho, out, g_chi, g_f, g_b


def _ctx(atm, model, prec):
    p = oracle.Problem(atm, model, *QUAD)
    return make_ctx(atm, model, *QUAD, prec, rho=oracle.initial_rho(p, atm))


def _cmp(g, o, tol, what, norm_tol=None):
    scale = np.max(np.abs(o))
    err = np.max(np.abs(g - o)) / scale
    assert err < tol, (what, err)
    if norm_tol is not None:
        rel = np.linalg.norm(g - o) / np.linalg.norm(o)
        assert rel < norm_tol, (what, rel)
    return err


@pytest.mark.parametrize("pol", [False, True])
def test_checkpointed_iterations_match_oracle_iterates(pol):
    atm, model = _case(pol)
    ctx = _ctx(atm, model, P.PORTA_FP64)
    ctx.iterate_ckpt(4, 3)
    f = np.asarray(atm["eps"]) * np.asarray(atm["bpl"])
    p = oracle.Problem(atm, model, *QUAD)
    ref = diff.iterate(p, oracle.initial_rho(p, atm), f, 4)
    got = ctx.get_rho()
    assert np.max(np.abs(got - ref) / np.abs(ref[..., :1])) < 1e-10


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
@pytest.mark.parametrize("pol", [False, True])
@pytest.mark.parametrize("niter,ckpt", [(1, 1), (3, 2), (4, 5)])
def test_iteration_gradients_match_oracle(prec, pol, niter, ckpt):
    atm, model = _case(pol)
    mu, az = synth.emergent_directions()
    gout = np.random.default_rng(17).normal(size=(len(mu), QUAD[2], atm["ny"], atm["nx"], 4 if pol else 1))
    rho, out_o, o_chi, o_f, o_b = _oracle(atm, model, niter, ckpt, mu, az, gout)
    ctx = _ctx(atm, model, prec)
    ctx.iterate_ckpt(niter, ckpt)
    out = np.zeros_like(gout)
    g_chi, g_f, g_b, out = ctx.iterate_vjp(mu, az, gout, out=out)
    fp64 = prec == P.PORTA_FP64
    tol = 1e-8 if fp64 else 2e-3
    _cmp(out, out_o, 1e-10 if fp64 else 1e-4, "out")
    _cmp(g_chi, o_chi, tol, "chi", None if fp64 else 2e-3)
    _cmp(g_f, o_f, tol, "f", None if fp64 else 2e-3)
    if pol:
        _cmp(g_b, o_b, tol, "B", None if fp64 else 2e-3)
    # rho is left at the last iterate
    got = ctx.get_rho()
    assert np.max(np.abs(got - rho) / np.abs(rho[..., :1])) < (1e-10 if fp64 else 1e-4)


@pytest.mark.parametrize("cluster,nu_group,tape_rays", [(1, 3, 1), (2, 2, 5), (3, 1, 7), (5, 2, 32)])
def test_launch_shapes_and_ray_batches_give_the_same_gradients(cluster, nu_group, tape_rays):
    """Forced adjoint shapes and a tape limit that splits the rays into batches
    (tape_rays rays per batch) against the default launch: the per-cluster
    accumulators differ in grouping only, so FP64 results agree to rounding."""
    atm, model = _case(True, nx=8, ny=6, nz=7, seed=5)
    mu, az = synth.emergent_directions()
    gout = np.random.default_rng(19).normal(size=(len(mu), QUAD[2], atm["ny"], atm["nx"], 4))
    ref_ctx = _ctx(atm, model, P.PORTA_FP64)
    ref_ctx.iterate_ckpt(2, 1)
    ref = ref_ctx.iterate_vjp(mu, az, gout)
    ctx = _ctx(atm, model, P.PORTA_FP64)
    ctx.set_adjoint_launch(cluster, nu_group)
    per_ray = QUAD[2] * atm["nx"] * atm["ny"] * atm["nz"] * 4 * 8
    ctx.set_tape_limit(tape_rays * per_ray)
    ctx.iterate_ckpt(2, 1)
    got = ctx.iterate_vjp(mu, az, gout)
    for g, r, what in zip(got, ref, ("chi", "f", "B")):
        _cmp(g, r, 1e-11, what)


def test_segment_store_and_per_step_rebuild_give_the_same_gradients():
    """Each checkpoint segment rebuilt once with its iterates kept on the device
    (the default) against every step back rebuilding its iterate from the
    checkpoint (a tape limit just below that store): the same iterates, so the
    FP64 gradients agree to the rounding of the different ray batches."""
    atm, model = _case(True, nx=8, ny=6, nz=7, seed=5)
    mu, az = synth.emergent_directions()
    gout = np.random.default_rng(29).normal(size=(len(mu), QUAD[2], atm["ny"], atm["nx"], 4))
    niter, ckpt = 6, 4
    ref_ctx = _ctx(atm, model, P.PORTA_FP64)
    ref_ctx.iterate_ckpt(niter, ckpt)
    ref = ref_ctx.iterate_vjp(mu, az, gout)
    ctx = _ctx(atm, model, P.PORTA_FP64)
    nvox = atm["nx"] * atm["ny"] * atm["nz"]
    store = ckpt * nvox * (6 + 6 + 1) * 8            # rho, J^K_Q and Lambda-bar* per iterate
    ctx.set_tape_limit(store - 8)
    ctx.iterate_ckpt(niter, ckpt)
    got = ctx.iterate_vjp(mu, az, gout)
    for g, r, what in zip(got, ref, ("chi", "f", "B")):
        _cmp(g, r, 1e-11, what)
    # the rebuild of the per-step path runs more formal solutions
    assert ctx.iterate_timing()["recompute_ms"] > ref_ctx.iterate_timing()["recompute_ms"]


def test_device_buffers_match_host_buffers():
    torch = pytest.importorskip("torch")
    atm, model = _case(True, seed=7)
    mu, az = synth.emergent_directions()
    gout = np.random.default_rng(23).normal(size=(len(mu), QUAD[2], atm["ny"], atm["nx"], 4))
    ctx = _ctx(atm, model, P.PORTA_FP32)
    ctx.iterate_ckpt(3, 2)
    host = ctx.iterate_vjp(mu, az, gout)
    dev = ctx.iterate_vjp(mu, az, torch.from_numpy(gout).cuda())
    for h, d in zip(host, dev):
        assert np.array_equal(h, d.cpu().numpy())


def test_iterate_vjp_needs_checkpoints():
    atm, model = _case(False)
    ctx = _ctx(atm, model, P.PORTA_FP64)
    mu, az = synth.emergent_directions()
    gout = np.zeros((len(mu), QUAD[2], atm["ny"], atm["nx"], 1))
    with pytest.raises(P.PortaError):
        ctx.iterate_vjp(mu, az, gout)
    with pytest.raises(P.PortaError):
        ctx.iterate_ckpt(0, 1)
