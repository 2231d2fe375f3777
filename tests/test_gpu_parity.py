"""Parity of the CUDA library (through the C ABI) with the FP64 oracle on the
same seeded inputs.

Tolerances (stated by the method's precision forms):
* FP64 sweep: 1e-10 relative (J^0_0, Lambda-bar*, Stokes I, rho); components
  that can vanish (J^2_Q, Q, U, V, S^2_Q) 1e-10 relative to the scalar they
  belong to (J^0_0, I, S^0_0).
* FP32 sweep: Stokes I 1e-5 relative; Q/I, U/I, V/I 1e-6 absolute. J^K_Q is a
  weighted sum of Stokes parameters with |T^K_Q| <= 1.1, so J^0_0 and
  Lambda-bar* get 1e-5 relative and J^2_Q 1e-5 J^0_0 absolute.
"""
import numpy as np
import pytest

import oracle
import paper_1307_4217_gb300 as P
from gpu_util import initial_rho, make_ctx, oracle_fs, polarized_case, unpolarized_case

pytestmark = pytest.mark.gpu

TOL = {P.PORTA_FP64: 1e-10, P.PORTA_FP32: 1e-5}


def _check_j(jg, lg, jo, lo, tol):
    s = np.abs(jo[..., :1])
    assert np.max(np.abs(jg[..., 0] - jo[..., 0]) / s[..., 0]) < tol
    if jo.shape[-1] > 1:
        assert np.max(np.abs(jg[..., 1:] - jo[..., 1:]) / s) < tol
    assert np.max(np.abs(lg - lo) / np.abs(lo)) < tol


def _check_stokes(Ig, Io, prec):
    I_o = Io[..., 0]
    scale = np.maximum(np.abs(I_o), 1e-300)
    tol = TOL[prec]
    assert np.max(np.abs(Ig[..., 0] - I_o) / scale) < tol
    if Io.shape[-1] > 1:
        ptol = 1e-10 if prec == P.PORTA_FP64 else 1e-6
        nz = np.abs(I_o) > 0
        assert np.max(np.abs(Ig[..., 1:][nz] / Ig[..., :1][nz] - Io[..., 1:][nz] / Io[..., :1][nz])) < ptol


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_unpolarized_box_formal_solution_and_see(prec):
    atm = unpolarized_case(16, 16, 32, seed=1)
    rho = initial_rho(atm, 0)
    rho[..., 0] *= np.exp(0.1 * np.sin(np.arange(rho[..., 0].size)).reshape(rho.shape[:-1]))
    ctx = make_ctx(atm, 0, 3, 8, 11, prec, rho=rho)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    p, (jo, lo) = oracle_fs(atm, 0, 3, 8, 11, rho)
    _check_j(jg, lg, jo, lo, TOL[prec])
    mc = ctx.see_update()
    rg = ctx.get_rho()
    ro, mco = oracle.see_update(p, jo, lo, rho)
    assert np.max(np.abs(rg - ro) / np.abs(ro)) < TOL[prec] * 10
    assert abs(mc - mco) <= TOL[prec] * 10 * max(1.0, mco)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_polarized_box_formal_solution(prec):
    atm = polarized_case(12, 10, 16, seed=3)
    rho = initial_rho(atm, 1, seed=4)
    ctx = make_ctx(atm, 1, 5, 16, 21, prec, rho=rho)
    ctx.formal_solve()
    jg, lg = ctx.accumulate_jkq()
    _, (jo, lo) = oracle_fs(atm, 1, 5, 16, 21, rho)
    _check_j(jg, lg, jo, lo, TOL[prec])


@pytest.mark.parametrize("cluster,nu_group", [(1, 6), (2, 5), (3, 4), (4, 3), (5, 7), (6, 3), (8, 2), (12, 2), (16, 7)])
def test_polarized_launch_shapes_agree(cluster, nu_group):
    """Every cluster size / frequency grouping gives the oracle's result; ny = 20 is
    not a multiple of 8 or 16 (ragged strips) and 21 frequencies leave a ragged pass."""
    atm = polarized_case(9, 20, 10, seed=5)
    rho = initial_rho(atm, 1, seed=6)
    ctx = make_ctx(atm, 1, 2, 4, 21, P.PORTA_FP64, cluster=cluster, nu_group=nu_group, rho=rho)
    ctx.formal_solve()
    info = ctx.launch_info()
    assert info["cluster"] == cluster
    jg, lg = ctx.accumulate_jkq()
    _, (jo, lo) = oracle_fs(atm, 1, 2, 4, 21, rho)
    _check_j(jg, lg, jo, lo, 1e-10)


def test_formal_solution_is_deterministic():
    atm = polarized_case(16, 16, 12, seed=7)
    ctx = make_ctx(atm, 1, 3, 8, 9, P.PORTA_FP32)
    out = []
    for _ in range(2):
        ctx.formal_solve()
        out.append(ctx.accumulate_jkq())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_probe_ray_stokes_vectors(prec):
    atm = polarized_case(8, 8, 12, seed=8)
    rho = initial_rho(atm, 1, seed=9)
    ctx = make_ctx(atm, 1, 3, 6, 7, prec, rho=rho)
    p = oracle.Problem(atm, 1, 3, 6, 7)
    for m in [0, 7, 17, 20, 35]:
        Ig, lg = ctx.probe_ray(m)
        for j in range(7):
            Io, lo = oracle.sweep_ray(p, rho, m, j)
            _check_stokes(Ig[j], Io, prec)
            assert np.max(np.abs(lg[j] - lo)) < TOL[prec]


def test_polarized_jacobi_iterations_fp64():
    atm = polarized_case(8, 8, 12, seed=10)
    ctx = make_ctx(atm, 1, 3, 8, 9, P.PORTA_FP64)
    p = oracle.Problem(atm, 1, 3, 8, 9)
    rho = oracle.initial_rho(p, atm)
    for it in range(3):
        ctx.formal_solve()
        ctx.accumulate_jkq(want=False)
        mc = ctx.see_update()
        jo, lo = oracle.formal_solve(p, rho)
        rho, mco = oracle.see_update(p, jo, lo, rho)
        rg = ctx.get_rho()
        s00 = np.abs(rho[..., :1])
        assert np.max(np.abs(rg - rho) / s00) < 1e-10, it
        assert abs(mc - mco) < 1e-9 * max(mco, 1e-3)


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
def test_emergent_stokes(prec):
    atm = polarized_case(10, 8, 14, seed=11)
    rho = initial_rho(atm, 1, seed=12)
    ctx = make_ctx(atm, 1, 2, 4, 9, prec, rho=rho)
    mu = np.array([1.0, 0.5, 0.5, 0.5, 0.5])
    chi = np.array([0.0, 0.0, np.pi / 2, np.pi, 1.5 * np.pi])
    og = ctx.emergent_stokes(mu, chi)
    p = oracle.Problem(atm, 1, 2, 4, 9)
    oo = oracle.emergent(p, rho, mu, chi)
    _check_stokes(og, oo, prec)


def test_edge_grids_fp64():
    """nx = ny = 1 (plane parallel), nz = 2 (boundary plus one plane), one frequency."""
    for (nx, ny, nz, nnu) in [(1, 1, 8, 5), (3, 1, 5, 3), (1, 4, 2, 1), (5, 3, 2, 2)]:
        atm = polarized_case(nx, ny, nz, seed=13)
        rho = initial_rho(atm, 1, seed=14)
        ctx = make_ctx(atm, 1, 2, 3, nnu, P.PORTA_FP64, rho=rho)
        ctx.formal_solve()
        jg, lg = ctx.accumulate_jkq()
        _, (jo, lo) = oracle_fs(atm, 1, 2, 3, nnu, rho)
        _check_j(jg, lg, jo, lo, 1e-10)


def test_call_order_and_invalid_inputs():
    atm = polarized_case(4, 4, 4, seed=15)
    ctx = P.Context(atm, 1, 2, 2, 3)
    with pytest.raises(P.PortaError) as e:
        ctx.formal_solve()
    assert e.value.code == P.PORTA_ESTATE
    bad = dict(atm)
    bad["chi"] = atm["chi"].copy()
    bad["chi"][1, 2, 3] = np.nan
    with pytest.raises(P.PortaError) as e:
        ctx.set_atmosphere(bad)
    assert e.value.code == P.PORTA_EINVAL
    bad = dict(atm)
    bad["eps"] = np.zeros_like(atm["eps"])
    with pytest.raises(P.PortaError) as e:
        ctx.set_atmosphere(bad)
    assert e.value.code == P.PORTA_EINVAL
    ctx.set_atmosphere(atm)
    with pytest.raises(P.PortaError) as e:
        ctx.accumulate_jkq()
    assert e.value.code == P.PORTA_ESTATE
    rho = initial_rho(atm, 1)
    rho[0, 0, 0, 0] = -1.0
    with pytest.raises(P.PortaError) as e:
        ctx.set_rho(rho)
    assert e.value.code == P.PORTA_EINVAL
    with pytest.raises(P.PortaError) as e:
        ctx.emergent_stokes([0.0], [0.0])
    assert e.value.code == P.PORTA_EINVAL
    ctx.set_rho(initial_rho(atm, 1))
    ctx.formal_solve()
    ctx.accumulate_jkq(want=False)
    assert ctx.see_update() > 0


def test_device_pointers_through_the_abi():
    torch = pytest.importorskip("torch")
    atm = polarized_case(8, 8, 8, seed=16)
    rho = initial_rho(atm, 1, seed=17)
    ctx = P.Context(atm, 1, 2, 4, 5, precision=P.PORTA_FP64)
    datm = {k: (torch.from_numpy(np.ascontiguousarray(v)).cuda() if isinstance(v, np.ndarray) and v.ndim == 3 else v)
            for k, v in atm.items()}
    ctx.set_atmosphere(datm)
    ctx.set_rho(torch.from_numpy(rho).cuda())
    ctx.formal_solve()
    jd = torch.zeros(rho.shape, dtype=torch.float64, device="cuda")
    ld = torch.zeros(rho.shape[:-1], dtype=torch.float64, device="cuda")
    ctx.accumulate_jkq(jd, ld)
    torch.cuda.synchronize()
    _, (jo, lo) = oracle_fs(atm, 1, 2, 4, 5, rho)
    _check_j(jd.cpu().numpy(), ld.cpu().numpy(), jo, lo, 1e-10)


def test_autotune_picks_a_valid_shape_and_keeps_parity():
    atm = polarized_case(16, 12, 10, seed=18)
    rho = initial_rho(atm, 1, seed=19)
    ctx = make_ctx(atm, 1, 2, 4, 9, P.PORTA_FP32, rho=rho)
    pick = ctx.autotune()
    assert 1 <= pick["cluster"] <= 16 and 1 <= pick["nu_group"] <= 9
    ctx.set_rho(rho)
    ctx.formal_solve()
    info = ctx.launch_info()
    assert (info["cluster"], info["nu_group"]) == (pick["cluster"], pick["nu_group"])
    jg, lg = ctx.accumulate_jkq()
    _, (jo, lo) = oracle_fs(atm, 1, 2, 4, 9, rho)
    _check_j(jg, lg, jo, lo, 1e-5)


def test_graph_iterations_match_eager_iterations():
    torch = pytest.importorskip("torch")
    atm = polarized_case(12, 10, 12, seed=25)
    rho = initial_rho(atm, 1, seed=26)
    eager = make_ctx(atm, 1, 3, 8, 9, P.PORTA_FP64, rho=rho)
    for _ in range(3):
        eager.formal_solve()
        eager.accumulate_jkq(want=False)
        mc_e = eager.see_update()
    graph = make_ctx(atm, 1, 3, 8, 9, P.PORTA_FP64, rho=rho)
    stream = torch.cuda.Stream()
    graph.set_stream(stream)
    mc_g = graph.run_iterations(1)
    mc_g = graph.run_iterations(2)
    assert mc_g == mc_e
    assert np.array_equal(graph.get_rho(), eager.get_rho())


@pytest.mark.parametrize("prec", [P.PORTA_FP64, P.PORTA_FP32])
@pytest.mark.parametrize("main,fill,frac", [((8, 7), (2, 3), 0.3), ((4, 21), (3, 5), 0.5), ((16, 7), (1, 2), 0.1)])
def test_concurrent_filler_launch(prec, main, fill, frac):
    """A second launch of a smaller shape over the cheapest fraction of the rays:
    oracle parity, and the dynamic work lists give the same bits on every call."""
    atm = polarized_case(9, 20, 10, seed=31)
    rho = initial_rho(atm, 1, seed=32)
    ctx = make_ctx(atm, 1, 2, 4, 21, prec, cluster=main[0], nu_group=main[1], rho=rho)
    ctx.set_fill(fill[0], fill[1], frac)
    assert ctx.fill_info() == {"cluster": fill[0], "nu_group": fill[1], "fraction": frac}
    out = []
    for _ in range(2):
        ctx.formal_solve()
        out.append(ctx.accumulate_jkq())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    _, (jo, lo) = oracle_fs(atm, 1, 2, 4, 21, rho)
    _check_j(out[0][0], out[0][1], jo, lo, TOL[prec])


def test_graph_iterations_with_filler_match_eager():
    torch = pytest.importorskip("torch")
    atm = polarized_case(12, 10, 12, seed=35)
    rho = initial_rho(atm, 1, seed=36)
    ctxs = []
    for _ in range(2):
        c = make_ctx(atm, 1, 3, 8, 9, P.PORTA_FP32, cluster=5, nu_group=9, rho=rho)
        c.set_fill(2, 3, 0.25)
        ctxs.append(c)
    eager, graph = ctxs
    for _ in range(3):
        eager.formal_solve()
        eager.accumulate_jkq(want=False)
        mc_e = eager.see_update()
    graph.set_stream(torch.cuda.Stream())
    graph.run_iterations(1)
    mc_g = graph.run_iterations(2)
    assert mc_g == mc_e
    assert np.array_equal(graph.get_rho(), eager.get_rho())
