"""The allocation-free formal solution (porta_formal_solve_noalloc) against the
regular entry points, through the C ABI on the GPU.

It serves callers that cannot allocate device memory (memory reserved up front
by another framework's pool, or loops that cannot afford cudaMalloc's implicit
synchronization). Its intermediates live in one fixed device array shared by
all calls, so two different problems are solved in a row and each must match
the regular path (FP32 sweeps: 1e-5 relative on J^0_0 and Lambda-bar*, 1e-5
J^0_0 on J^2_Q, the tolerances of the other FP32 parity tests). The file is
named to be collected last."""
import numpy as np
import pytest

import paper_1307_4217_gb300 as P
from gpu_util import initial_rho, make_ctx, polarized_case, unpolarized_case

pytestmark = pytest.mark.gpu


def _regular(atm, model, quad, rho):
    ctx = make_ctx(atm, model, *quad, P.PORTA_FP32, rho=rho)
    ctx.formal_solve()
    j, l = ctx.accumulate_jkq()
    ctx.close()
    return j, l


def _noalloc(atm, model, quad, rho):
    import torch
    datm = {k: torch.from_numpy(np.ascontiguousarray(atm[k], dtype=np.float64)).cuda()
            for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz") if atm.get(k) is not None}
    drho = torch.from_numpy(np.ascontiguousarray(rho)).cuda()
    nj = 1 if model == 0 else 6
    shape = (atm["nz"], atm["ny"], atm["nx"])
    dj = torch.full(shape + (nj,), float("nan"), dtype=torch.float64, device="cuda")
    dl = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = P.porta_formal_solve_noalloc(atm, model, *quad, 4.0, datm, drho.data_ptr(), dj.data_ptr(), dl.data_ptr())
    torch.cuda.synchronize()
    assert rc == P.PORTA_OK, rc
    return dj.cpu().numpy(), dl.cpu().numpy()


def _close(a, b):
    jn, ln = a
    jr, lr = b
    s = np.abs(jr[..., :1])
    assert np.max(np.abs(jn - jr) / s) < 1e-5
    assert np.max(np.abs(ln - lr) / np.abs(lr)) < 1e-5


def test_noalloc_matches_regular_path_on_two_calls_in_a_row():
    pytest.importorskip("torch")
    atm1 = polarized_case(12, 10, 16, seed=21)
    rho1 = initial_rho(atm1, 1, seed=22)
    q1 = (5, 16, 21)
    atm2 = unpolarized_case(16, 16, 32, seed=23)
    rho2 = initial_rho(atm2, 0)
    q2 = (3, 8, 11)
    ref1 = _regular(atm1, 1, q1, rho1)
    ref2 = _regular(atm2, 0, q2, rho2)
    _close(_noalloc(atm1, 1, q1, rho1), ref1)      # first call (sets the scratch address up)
    _close(_noalloc(atm2, 0, q2, rho2), ref2)      # second call, different problem, reused scratch
    _close(_noalloc(atm1, 1, q1, rho1), ref1)


def test_noalloc_rejects_problems_beyond_its_scratch():
    pytest.importorskip("torch")
    atm = polarized_case(64, 64, 16, seed=24)     # 65536 voxels x 160 rays >> 32 MiB
    rho = initial_rho(atm, 1)
    import torch
    datm = {k: torch.from_numpy(np.ascontiguousarray(atm[k])).cuda() for k in ("chi", "eps", "bpl", "vel", "bx", "by", "bz")}
    drho = torch.from_numpy(rho).cuda()
    out = torch.zeros(rho.shape, dtype=torch.float64, device="cuda")
    ls = torch.zeros(rho.shape[:-1], dtype=torch.float64, device="cuda")
    rc = P.porta_formal_solve_noalloc(atm, 1, 5, 16, 21, 4.0, datm, drho.data_ptr(), out.data_ptr(), ls.data_ptr())
    assert rc == P.PORTA_ESCRATCH
    assert float(out.abs().max()) == 0.0
