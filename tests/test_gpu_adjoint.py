"""Adjoint of the emergent Stokes profiles on the GPU (porta_emergent_vjp and
the torch.autograd.Function around it) against the oracle's FP64 adjoint and
central finite differences of the FP64 forward solution.

Tolerances. FP64: the GPU and the oracle evaluate the same derivatives in a
different order and form (the oracle reverses a general 4x4 solve), so the
gradients agree to rounding amplified by the sums over directions and
frequencies: 1e-9 of the largest gradient component. FP32: the forward
Stokes vectors carry 1e-5 relative error and every gradient term is a product
of a few such factors, summed over up to 9 nodes x frequencies x directions in
FP32 per node and in FP64 across groups: 1e-3 of the largest component and
1e-3 in the relative 2-norm. The B gradient is the least accurate: in
optically thick layers its eta_V (absorption) and eps_V (emission) terms
nearly cancel (their sum is proportional to S^0_0 - I), which amplifies the
FP32 rounding of each (2e-4 in the 2-norm on the small grids here). Against
central differences (relative step 1e-4, FP64 forward) the FP32 adjoint
agrees to 1e-3 relative.
"""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
import synth
from gpu_util import initial_rho, make_ctx

pytestmark = pytest.mark.gpu


def _case(nx, ny, nz, seed, pol=True):
    if pol:
        atm = synth.random_box(nx, ny, nz, seed=seed)
        for k in ("bx", "by", "bz"):
            atm[k] = atm[k] * 30.0      # Zeeman term visible at these sizes
    else:
        atm = synth.plane_parallel_box(nx, ny, nz, modulation=0.3)
        rng = np.random.default_rng(seed)
        atm["vel"] = 0.7 * rng.normal(size=atm["chi"].shape)
    model = 1 if pol else 0
    rho = initial_rho(atm, model, seed=seed + 1 if pol else None)
    if not pol:
        # a varying source function: with S constant every control point lies on
        # the step-2 boundary of BESSER (d_M = d_P = 0), where the map has a kink
        rho[..., 0] *= np.exp(0.2 * np.random.default_rng(seed + 1).normal(size=rho.shape[:-1]))
    return atm, model, rho


def _oracle_grads(atm, model, rho, n_nu, mu, az, gout):
    p = oracle.Problem(atm, model, 1, 1, n_nu)
    return oracle.emergent_vjp(p, rho, mu, az, gout)


def _cmp(g, o, tol, what):
    scale = np.max(np.abs(o))
    err = np.max(np.abs(g - o)) / scale
    assert err < tol, (what, err)
    return err


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
@pytest.mark.parametrize("cluster,nu_group", [(0, 0), (1, 5), (2, 2), (3, 1), (5, 3), (10, 4)])
def test_polarized_adjoint_matches_oracle(prec, cluster, nu_group):
    nx, ny, nz, n_nu = 12, 10, 9, 5
    atm, model, rho = _case(nx, ny, nz, seed=11)
    mu, az = synth.emergent_directions()
    ctx = make_ctx(atm, model, 1, 1, n_nu, prec, rho=rho)
    ctx.set_adjoint_launch(cluster, nu_group)
    out_shape = (len(mu), n_nu, ny, nx, 4)
    gout = np.random.default_rng(4).normal(size=out_shape)
    out = np.zeros(out_shape)
    g_chi, g_e, g_b, out = ctx.emergent_vjp(mu, az, gout, out=out)
    info = ctx.adjoint_info()
    if cluster:
        assert info["cluster"] == cluster and info["nu_group"] == nu_group
    o_chi, o_e, o_b = _oracle_grads(atm, model, rho, n_nu, mu, az, gout)
    tol = 1e-9 if prec == P.PORTA_FP64 else 1e-3
    _cmp(g_chi, o_chi, tol, "chi")
    _cmp(g_e, o_e, tol, "e")
    _cmp(g_b, o_b, tol, "B")
    if prec == P.PORTA_FP32:
        for g, o in ((g_chi, o_chi), (g_e, o_e), (g_b, o_b)):
            assert np.linalg.norm(g - o) / np.linalg.norm(o) < 1e-3
    # the forward output of the same call is the emergent Stokes vector
    ref = ctx.emergent_stokes(mu, az)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_unpolarized_adjoint_matches_oracle(prec):
    nx, ny, nz, n_nu = 9, 7, 8, 4
    atm, model, rho = _case(nx, ny, nz, seed=5, pol=False)
    mu = np.array([1.0, 0.45, 0.8])
    az = np.array([0.0, 2.2, 4.0])
    ctx = make_ctx(atm, model, 1, 1, n_nu, prec, rho=rho)
    gout = np.random.default_rng(6).normal(size=(len(mu), n_nu, ny, nx, 1))
    g_chi, g_e, _ = ctx.emergent_vjp(mu, az, gout)
    o_chi, o_e, _ = _oracle_grads(atm, model, rho, n_nu, mu, az, gout)
    tol = 1e-9 if prec == P.PORTA_FP64 else 1e-3
    _cmp(g_chi, o_chi, tol, "chi")
    _cmp(g_e, o_e, tol, "e")


def test_fp32_adjoint_where_the_profile_floor_is_reached():
    # large velocity shifts put |x - s| beyond the FP32 profile floor exp(-60):
    # optical paths of 1e-28 and their reciprocals must stay finite
    nx, ny, nz, n_nu = 8, 6, 12, 7
    atm = synth.random_box(nx, ny, nz, seed=21, sigma_v=4.0)
    rho = initial_rho(atm, 1, seed=22)
    mu, az = synth.emergent_directions()
    gout = np.random.default_rng(3).normal(size=(len(mu), n_nu, ny, nx, 4))
    o = _oracle_grads(atm, 1, rho, n_nu, mu, az, gout)
    ctx = make_ctx(atm, 1, 1, 1, n_nu, P.PORTA_FP32, rho=rho)
    g = ctx.emergent_vjp(mu, az, gout)
    for a, b, what in zip(g, o, ("chi", "e", "B")):
        assert np.all(np.isfinite(a)), what
        _cmp(a, b, 1e-3, what)


def test_adjoint_edge_sizes_and_determinism():
    # two planes, a single row and a single column, and a cluster as large as ny
    mu, az = synth.emergent_directions()
    for nx, ny, nz, cl in ((5, 4, 2, 4), (1, 6, 5, 3), (7, 1, 4, 1)):
        atm, model, rho = _case(nx, ny, nz, seed=2)
        ctx = make_ctx(atm, model, 1, 1, 3, P.PORTA_FP64, rho=rho)
        ctx.set_adjoint_launch(cl, 0)
        gout = np.random.default_rng(1).normal(size=(len(mu), 3, ny, nx, 4))
        g = ctx.emergent_vjp(mu, az, gout)
        o = _oracle_grads(atm, model, rho, 3, mu, az, gout)
        for a, b in zip(g, o):
            _cmp(a, b, 1e-9, (nx, ny, nz))
        g2 = ctx.emergent_vjp(mu, az, gout)
        for a, b in zip(g, g2):
            assert np.array_equal(a, b)


def test_autograd_function_matches_vjp_and_directional_difference():
    import torch
    from paper_1307_4217_gb300.autograd import emergent_stokes
    nx, ny, nz, n_nu = 8, 8, 7, 3
    atm, model, rho = _case(nx, ny, nz, seed=9)
    dev = torch.device("cuda:0")
    mu, az = synth.emergent_directions()
    ctx = make_ctx(atm, model, 1, 1, n_nu, P.PORTA_FP64, rho=rho)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    fixed = {"vel": t(atm["vel"]), "bpl": t(atm["bpl"]), "eps": t(atm["eps"]), "ratios": t(rho / rho[..., :1])}
    chi = t(atm["chi"]).requires_grad_()
    e = t(atm["chi"] * rho[..., 0]).requires_grad_()
    B = t(np.stack([atm["bx"], atm["by"], atm["bz"]])).requires_grad_()
    target = torch.randn((len(mu), n_nu, ny, nx, 4), dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(3))
    out = emergent_stokes(ctx, fixed, mu, az, chi, e, B)
    loss = ((out - target) ** 2).sum()
    loss.backward()
    gout = (2 * (out - target)).detach().cpu().numpy()
    g = ctx.emergent_vjp(mu, az, gout)
    for a, b in zip((chi.grad, e.grad, B.grad), g):
        assert np.allclose(a.cpu().numpy(), b, rtol=1e-12, atol=0)
    # directional central difference of the loss in FP64
    rng = np.random.default_rng(0)
    dirs = [t(rng.normal(size=x.shape)) * x.detach() for x in (chi, e, B)]
    h = 1e-6

    def L(s):
        with torch.no_grad():
            o = emergent_stokes(ctx, fixed, mu, az, chi + s * dirs[0], e + s * dirs[1], B + s * dirs[2])
            return float(((o - target) ** 2).sum())
    fd = (L(h) - L(-h)) / (2 * h)
    an = sum(float((x.grad * dx).sum()) for x, dx in zip((chi, e, B), dirs))
    assert abs(fd - an) <= 1e-5 * abs(an)


@pytest.mark.slow
def test_full_size_fp32_adjoint_matches_central_differences():
    """64^3 polarized box, 21 frequencies, vertical + 4 oblique emergent rays;
    loss = sum of squared IQUV differences from the seed+1 model's profiles."""
    atm = synth.random_box(64, 64, 64, seed=0)
    tgt_atm = synth.random_box(64, 64, 64, seed=1)
    model, n_nu = 1, 21
    rho = initial_rho(atm, model, seed=7)
    mu, az = synth.emergent_directions()
    c64 = make_ctx(tgt_atm, model, 5, 16, n_nu, P.PORTA_FP64, rho=initial_rho(tgt_atm, model, seed=8))
    target = c64.emergent_stokes(mu, az)
    c64.set_atmosphere(atm)
    c64.set_rho(rho)
    c32 = make_ctx(atm, model, 5, 16, n_nu, P.PORTA_FP32, rho=rho)
    out32 = c32.emergent_stokes(mu, az)
    out64 = c64.emergent_stokes(mu, az)
    g32 = c32.emergent_vjp(mu, az, 2 * (out32 - target))
    g64 = c64.emergent_vjp(mu, az, 2 * (out64 - target))
    chi0, e0 = atm["chi"], atm["chi"] * rho[..., 0]
    B0 = np.stack([atm["bx"], atm["by"], atm["bz"]])
    ratios = rho / rho[..., :1]

    def emergent_at(chi, e, B):
        a = dict(atm)
        a.update(chi=chi, bx=B[0], by=B[1], bz=B[2])
        c64.set_atmosphere(a)
        c64.set_rho(ratios * (e / chi)[..., None])
        return c64.emergent_stokes(mu, az)

    rng = np.random.default_rng(123)
    picks = [tuple(int(rng.integers(0, s)) for s in (64, 64, 64)) for _ in range(64)]
    # voxels deep below the surface have gradients many orders below the largest;
    # there agreement is measured against 1e-3 of the largest gradient of the parameter
    floor = {"chi": 1e-3 * np.max(np.abs(g64[0])), "e": 1e-3 * np.max(np.abs(g64[1])),
             "bx": 1e-3 * np.max(np.abs(g64[2])), "by": 1e-3 * np.max(np.abs(g64[2])),
             "bz": 1e-3 * np.max(np.abs(g64[2]))}
    kept = rejected = 0
    worst32 = worst64 = 0.0
    for v in picks:
        for name in ("chi", "e", "bx", "by", "bz"):
            if name == "chi":
                x0, gi, gd = chi0[v], g32[0][v], g64[0][v]
            elif name == "e":
                x0, gi, gd = e0[v], g32[1][v], g64[1][v]
            else:
                c = "xyz".index(name[1])
                x0, gi, gd = B0[(c,) + v], g32[2][(c,) + v], g64[2][(c,) + v]
            step = 1e-4 * (abs(x0) if name in ("chi", "e") else np.linalg.norm(B0[(slice(None),) + v]))

            def o_at(dx):
                chi, e, B = chi0.copy(), e0.copy(), B0.copy()
                if name == "chi":
                    chi[v] += dx
                elif name == "e":
                    e[v] += dx
                else:
                    B[(c,) + v] += dx
                return emergent_at(chi, e, B)

            def cd(h):
                # L(+h) - L(-h) for the quadratic loss, without forming L (whose
                # rounding would swamp the change made by one deep voxel)
                op, om = o_at(h), o_at(-h)
                return float(np.sum((op - om) * (op + om - 2 * target))) / (2 * h)

            fd = cd(step)
            ref = max(abs(fd), floor[name])
            ok32 = abs(gi - fd) <= 1e-3 * ref
            ok64 = abs(gd - fd) <= 1e-4 * ref
            if not (ok32 and ok64):
                fd2 = cd(step / 2)
                if abs(fd2 - fd) > 1e-5 * ref:
                    rejected += 1       # a branch of the control point changes within the step
                    continue
            assert ok32, (v, name, gi, fd)
            assert ok64, (v, name, gd, fd)
            worst32 = max(worst32, abs(gi - fd) / ref)
            worst64 = max(worst64, abs(gd - fd) / ref)
            kept += 1
    print(f"central differences at 64 voxels x 5 parameters: kept {kept}, rejected {rejected}, "
          f"worst relative error FP32 {worst32:.2e}, FP64 {worst64:.2e}")
    assert kept >= 0.9 * 64 * 5, (kept, rejected)


@pytest.mark.slow
def test_full_size_adjoint_matches_cpu_oracle_adjoint_on_one_direction():
    """64^3 box, 21 frequencies, the vertical and one oblique direction: FP32 and
    FP64 GPU adjoints against the oracle's FP64 adjoint (a bounded CPU sample)."""
    atm = synth.random_box(64, 64, 64, seed=0)
    model, n_nu = 1, 21
    rho = initial_rho(atm, model, seed=7)
    mu, az = np.array([1.0, 0.5]), np.array([0.0, 0.5 * np.pi])
    gout = np.random.default_rng(2).normal(size=(2, n_nu, 64, 64, 4))
    o = _oracle_grads(atm, model, rho, n_nu, mu, az, gout)
    for prec, tol in ((P.PORTA_FP64, 1e-9), (P.PORTA_FP32, 1e-3)):
        ctx = make_ctx(atm, model, 5, 16, n_nu, prec, rho=rho)
        g = ctx.emergent_vjp(mu, az, gout)
        for a, b, what in zip(g, o, ("chi", "e", "B")):
            _cmp(a, b, tol, what)
