"""The five-level polarized atom at the full multilevel workload size
(128 x 128 x 96, four lines x 31 frequencies, 160 rays, FP32 sweeps, the
autotuned launch the benchmark times): properties that hold at any size on
every voxel, and the oracle's update of sampled voxels from the same inputs.

* the trace sum_J sqrt(2J+1) rho^0_0(J) = 1 and positive populations;
* the update of 64 random voxels, recomputed by the oracle from the GPU's
  radiation tensors (J^K_Q, K = 0, 1, 2), Lambda-bar* and old multipoles, to
  1e-11 of the largest unknown (the update runs in FP64 on both sides);
* orientation (K = 1) present in J^1_Q and in the updated multipoles.
"""
import numpy as np
import pytest

import paper_1307_4217_gb300 as P
import synth
from oracle import ml, mlpol

pytestmark = pytest.mark.gpu


def test_full_size_update_matches_oracle_on_sampled_voxels():
    import torch
    nx, ny, nz = 128, 128, 96
    atm = synth.multilevel_box(nx, ny, nz, seed=0)
    atom = synth.multilevel_atom(seed=0)
    tab = mlpol.Tables(atom)
    pops0 = ml.lte_populations(atom, atm["kT"])
    ctx = P.MlContext(atm, atom, 5, 16, 31, precision=P.PORTA_FP32, polarized=True, zeta=1e-5)
    s = torch.cuda.Stream()
    ctx.set_stream(s)
    ctx.set_atmosphere(atm)
    ctx.set_pops(pops0)
    with torch.cuda.stream(s):
        ctx.autotune()
        ctx.set_pops(pops0)
        ctx.ml_iterate(2)                        # a state with atomic polarization
        x0 = ctx.get_unknowns()
        jb, ls = ctx.ml_formal_solve()
        ctx.ml_see_update()
        x1 = ctx.get_unknowns()
    s.synchronize()
    pops = tab.populations(x1)
    assert np.min(pops) > 0
    assert np.max(np.abs(pops.sum(-1) - 1)) < 1e-12
    rng = np.random.default_rng(0)
    idx = rng.choice(nx * ny * nz, 64, replace=False)
    flat = lambda a: a.reshape((nz * ny * nx,) + a.shape[3:])
    j9 = np.moveaxis(jb, 0, -2)
    bv = np.stack([atm["bx"], atm["by"], atm["bz"]], -1)
    want, _ = mlpol.see_update(tab, flat(atm["kT"])[idx], flat(x0)[idx], flat(j9)[idx],
                               flat(np.moveaxis(ls, 0, -1))[idx], flat(bv)[idx])
    got = flat(x1)[idx]
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))
    rb = mlpol.real_basis(atom)
    assert np.max(np.abs(x1[..., rb.index((3, 2, 0, 0))])) > 0
    # orientation from the circular polarization of the Zeeman effect (J^1_Q from Stokes V)
    assert np.max(np.abs(jb[..., 1:4])) > 0
    assert np.max(np.abs(x1[..., rb.index((3, 1, 0, 0))])) > 0
