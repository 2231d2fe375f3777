#!/usr/bin/env python
"""Benchmark of the PORTA formal-solver hot path on GB300.

Workload: the polarized two-level atom (Jl = 0 -> Ju = 1; scattering
polarization, Hanle and weak-field Zeeman effects) in a 64x64x64 random box,
160 rays (5 Gauss inclinations per hemisphere x 16 azimuths) and 21
frequencies. One step = one Jacobi iteration through the C ABI:
porta_formal_solve (FP32 sweeps, fused frequency integration) +
porta_accumulate_jkq (FP64 J^K_Q, Lambda-bar*) + porta_see_update (FP64
Hanle SEE and residual). The metric is voxel.ray.frequency updates per second
of the formal solution (64^3 x 160 x 21 = 8.8e8 updates per step).

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "polarized SC formal-solver voxel·ray·freq updates/s; % roofline; FP32 vs FP64"
UNIT = "updates/s"
NX = NY = NZ = 64
N_MU, N_CHI, N_NU = 5, 16, 21
NRAY = 2 * N_MU * N_CHI
ML_ZETA = 1e-5          # Zeeman splitting per gauss (Doppler widths) of the multilevel lines
UPDATES = NX * NY * NZ * NRAY * N_NU
WORKLOAD = ("polarized two-level atom (Jl=0->Ju=1, Hanle + weak-field Zeeman), random box 64x64x64, "
            "160 rays, 21 frequencies; one Jacobi iteration per step (FP32 sweeps, FP64 SEE)")
# algorithmic floating-point operations per voxel.ray.frequency update of the
# formal solution, counted stage by stage with each node's transfer coefficients
# once per ray and frequency: node coefficients, bilinear interpolation at M and
# P, source functions and optical paths 140, exponential-integral coefficients 25,
# BESSER control points for the 4 Stokes parameters 72, right-hand side of Eq. 7
# 34, the I-V coupling solve 9, Lambda* and the frequency accumulation 11, the
# J^K_Q finalize per (ray, voxel) spread over 21 frequencies 2
F_ALG = 293
# FP32 issue peak of the GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz
SMS, LANES, SM_MAX_MHZ = 152, 128, 2070.0
PEAK_FP32_TFLOPS = SMS * LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_pol64_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1307_4217_gb300", "csrc", f)
                  for f in ("sweep.cu", "sweep_common.cuh", "device_math.cuh", "porta_internal.cuh")]


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_traffic():
    """DRAM bytes per sweep launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        d = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != kernel_hash():
        return None
    return d.get("dram_bytes_per_launch")


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-rays", type=int, default=4)
    ap.add_argument("--adjoint-reps", type=int, default=5,
                    help="timed calls of the emergent-Stokes adjoint (0 skips it)")
    ap.add_argument("--mg-cycles", type=int, default=3, help="timed multigrid V-cycles (0 skips them)")
    ap.add_argument("--iter-adjoint", default="20,5",
                    help="gradients through Jacobi iterations: 'iterations,checkpoint spacing' (0 skips them)")
    ap.add_argument("--ml-steps", type=int, default=3,
                    help="timed Jacobi iterations of the multilevel atom on the 128x128x96 grid (0 skips them)")
    ap.add_argument("--ml-mg-cycles", type=int, default=3, help="timed multigrid V-cycles of the multilevel atom")
    ap.add_argument("--mlpol-mg-cycles", type=int, default=1,
                    help="timed multigrid V-cycles of the polarized multilevel atom")
    ap.add_argument("--ml-grid", default="128,128,96",
                    help="grid of the multilevel workloads nx,ny,nz (a smaller one for profiling captures)")
    ap.add_argument("--mlpol-steps", type=int, default=2,
                    help="timed Jacobi iterations of the polarized multilevel atom on 128x128x96 (0 skips them)")
    ap.add_argument("--fill", default="", help="force the concurrent filler launch: cluster,nu_group,fraction")
    ap.add_argument("--adjoint-cluster", type=int, default=0, help="force the adjoint cluster size (skips its tuning)")
    ap.add_argument("--adjoint-nu-group", type=int, default=0, help="force the adjoint frequencies per pass")
    ap.add_argument("--cluster", type=int, default=0, help="force the sweep cluster size (skips the autotuner)")
    ap.add_argument("--nu-group", type=int, default=0, help="force frequencies per pass (skips the autotuner)")
    ap.add_argument("--workload", choices=["pol64", "batched256"], default="pol64",
                    help="pol64: the 64^3 polarized box (default); batched256: 256 uneven boxes in one launch")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(values, device):
    """Element-wise maximum over ranks of per-rank timings: the slowest replica
    sets the job's time (an all-reduce on timings only, never on solver data)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank, world, seconds):
    """Whole-job rate: every rank solves its own replica of the workload."""
    return world * units_per_rank / seconds


# ---------------------------------------------------------------- clocks sampling

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append(dict(sm=float(p[1]), smax=float(p[2]), reasons=p[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for n, v in zip(names[1:], r["reasons"][1:]):
                if v.lower() == "active":
                    seen.add(n)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(seen), "samples": len(rows)}


# ---------------------------------------------------------------- CPU baseline (oracle)

def oracle_sample(nrays, seed=0):
    """Time the FP64 oracle on `nrays` full rays (all 21 frequencies, the whole 64^3 box)."""
    import oracle
    atm = synth.random_box(NX, NY, NZ, seed=seed)
    p = oracle.Problem(atm, oracle.MODEL_HANLE, N_MU, N_CHI, N_NU)
    rho = oracle.initial_rho(p, atm)
    rays = np.linspace(0, NRAY - 1, nrays).astype(int)
    t0 = time.perf_counter()
    for m in rays:
        oracle.formal_solve(p, rho, rays_range=(int(m), int(m) + 1))
    dt = time.perf_counter() - t0
    n = nrays * NX * NY * NZ * N_NU
    return n / dt, dt, f"{nrays} rays x 21 frequencies over the full 64^3 box ({n} updates, {dt:.1f} s)"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    atm = synth.random_box(NX, NY, NZ, seed=0)
    p = oracle.Problem(atm, oracle.MODEL_HANLE, N_MU, N_CHI, N_NU)
    rho = oracle.initial_rho(p, atm)
    per_step = NX * NY * NZ * N_NU      # one ray, all frequencies, per step
    for s in range(args.warmup):
        oracle.formal_solve(p, rho, rays_range=(s % NRAY, s % NRAY + 1))
    t0 = time.perf_counter()
    for s in range(args.steps):
        m = (args.warmup + s * 37) % NRAY
        oracle.formal_solve(p, rho, rays_range=(m, m + 1))
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_step": "one ray x 21 frequencies over the full 64^3 box"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} rays x 21 frequencies over the full 64^3 box"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- workloads

class Workload:
    """A benchmarked problem: its context factory, update count per formal
    solution, and the oracle sample used for the CPU baseline."""

    def __init__(self, name, rank):
        import paper_1307_4217_gb300 as P
        self.name = name
        if name == "pol64":
            self.atm = synth.random_box(NX, NY, NZ, seed=rank)
            self.quad = (N_MU, N_CHI, N_NU)
            self.updates = UPDATES
            self.desc = WORKLOAD
            self.rho0 = np.zeros((NZ, NY, NX, 6))
            self.rho0[..., 0] = self.atm["bpl"]
            self.config = {"grid": [NX, NY, NZ], "rays": NRAY, "frequencies": N_NU}
        elif name == "batched256":
            self.atms = synth.batched_boxes(256, seed=rank)
            self.quad = (4, 10, 21)
            nvox = sum(a["nx"] * a["ny"] * a["nz"] for a in self.atms)
            self.updates = nvox * 80 * 21
            self.desc = ("256 independent polarized two-level boxes (Nx = Ny in {8,16,24,32,48}, Nz in 16..64, "
                         "own seeds), 80 rays, 21 frequencies; one Jacobi iteration of all boxes per step "
                         "(one persistent sweep launch, FP32 sweeps, FP64 SEE)")
            self.rho0 = np.concatenate([np.stack([a["bpl"].ravel()] + [np.zeros(a["bpl"].size)] * 5, axis=1)
                                        for a in self.atms])
            self.config = {"boxes": 256, "voxels": nvox, "rays": 80, "frequencies": 21}
        else:
            raise ValueError(name)
        self.P = P

    def context(self, precision, cluster, nu_group):
        P = self.P
        if self.name == "pol64":
            ctx = P.Context(self.atm, P.PORTA_MODEL_TWOLEVEL_HANLE, *self.quad, precision=precision,
                            cluster=cluster, nu_group=nu_group)
            ctx.set_atmosphere(self.atm)
        else:
            ctx = P.BatchContext(self.atms, P.PORTA_MODEL_TWOLEVEL_HANLE, *self.quad, precision=precision,
                                 cluster=cluster, nu_group=nu_group)
            ctx.set_atmosphere(self.atms)
        ctx.set_rho(self.rho0)
        return ctx

    def oracle_sample(self, nrays):
        import oracle
        if self.name == "pol64":
            return oracle_sample(nrays)
        # a few boxes of the batch, all rays and frequencies
        t0 = time.perf_counter()
        n = 0
        for b in (0, 85, 170):
            a = self.atms[b]
            p = oracle.Problem(a, oracle.MODEL_HANLE, *self.quad)
            oracle.formal_solve(p, oracle.initial_rho(p, a))
            n += a["nx"] * a["ny"] * a["nz"] * 80 * 21
        dt = time.perf_counter() - t0
        return n / dt, dt, f"boxes 0, 85, 170 of the batch, all rays and frequencies ({n} updates, {dt:.1f} s)"


# ---------------------------------------------------------------- GPU arm

def run_cuda(args):
    import torch
    import paper_1307_4217_gb300 as P
    from paper_1307_4217_gb300 import build as B

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()

    # Each rank solves its own problem (independent replicas: weak scaling, no data-path collective).
    wl = Workload(args.workload, rank)
    stream = torch.cuda.Stream(device=dev)
    forced = args.cluster > 0 or args.nu_group > 0

    def make(precision):
        ctx = wl.context(precision, args.cluster, args.nu_group)
        ctx.set_stream(stream)
        if not forced:
            ctx.autotune()          # launch-shape autotuner (outside the timed region)
            ctx.set_rho(wl.rho0)
        if args.fill:
            cl, nu, fr = args.fill.split(",")
            ctx.set_fill(int(cl), int(nu), float(fr))
        return ctx

    ctx = make(P.PORTA_FP32)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        # warm-up: eager calls, then the captured graph of one Jacobi iteration
        for _ in range(args.warmup):
            ctx.formal_solve()
            ctx.accumulate_jkq(want=False)
            ctx.see_update(residual=False)
        ctx.run_iterations(1, residual=False)
        barrier()
        # timed steps: one graph replay (formal solution, J^K_Q sums, SEE, residual) each
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        sampler = ClockSampler(local)
        sampler.start()
        barrier()
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            ctx.run_iterations(1, residual=False)
            ev[k][1].record(stream)
        barrier()
        clocks = sampler.stop()
        step_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
        # sweep kernel alone (eager formal solutions), for the roofline
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            ctx.formal_solve()
            evs[k][1].record(stream)
        barrier()
        sweep_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    info = ctx.launch_info()
    fill = ctx.fill_info()

    # end to end through the ABI with pinned host buffers: rho in, one iteration, rho and residual out
    rho_h = torch.from_numpy(wl.rho0.copy()).pin_memory()
    rho_out = torch.empty_like(rho_h).pin_memory()
    with torch.cuda.stream(stream):
        ctx.set_rho(rho_h)
        ctx.run_iterations(1)
        ctx.get_rho(rho_out)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_rho(rho_h)
            residual = ctx.run_iterations(1)
            ctx.get_rho(rho_out)
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = rho_h.numel() * 8
    d2h = rho_out.numel() * 8 + 8

    # FP64 plain form of the same step (single box only: the FP64 batch takes ~15 s per step)
    fp64 = None
    if args.fp64_steps > 0 and wl.name == "pol64":
        ctx64 = make(P.PORTA_FP64)
        with torch.cuda.stream(stream):
            ctx64.run_iterations(1, residual=False)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx64.run_iterations(args.fp64_steps, residual=False)
            e1.record(stream)
            barrier()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        fp64 = {"value": world * wl.updates / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "dtype": "f64",
                "launch": ctx64.launch_info()}
        ctx64.close()

    # reverse mode of the emergent Stokes profiles (differentiation workload: the
    # same 64^3 box, vertical + 4 oblique emergent rays, all frequencies), FP32:
    # device time of the forward sweep with its tape and of the adjoint sweep
    adjoint = None
    if args.adjoint_reps > 0 and wl.name == "pol64":
        mu, az = synth.emergent_directions()
        nz, ny, nx = ctx.shape
        gen = torch.Generator(device=dev).manual_seed(1234)
        gout = torch.randn((len(mu), ctx.nnu, ny, nx, ctx.ns), dtype=torch.float64, device=dev, generator=gen)
        gbuf = [torch.empty((nz, ny, nx), dtype=torch.float64, device=dev) for _ in range(2)]
        gbuf.append(torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev))
        ts = []
        with torch.cuda.stream(stream):
            ctx.set_rho(wl.rho0)
            ctx.set_adjoint_launch(args.adjoint_cluster, args.adjoint_nu_group)
            ctx.emergent_vjp(mu, az, gout, g_chi=gbuf[0], g_e=gbuf[1], g_b=gbuf[2])   # shape tuning
            for _ in range(args.adjoint_reps):
                ctx.emergent_vjp(mu, az, gout, g_chi=gbuf[0], g_e=gbuf[1], g_b=gbuf[2])
                ts.append(ctx.adjoint_timing())
        f_ms = float(np.median([t["forward_ms"] for t in ts]))
        a_ms = float(np.median([t["adjoint_ms"] for t in ts]))
        nupd = len(mu) * ctx.nnu * nx * ny * nz
        adjoint = {"workload": f"{nx}x{ny}x{nz} polarized, {ctx.nnu} frequencies, vertical + 4 oblique (mu=0.5) "
                               "emergent rays; gradients w.r.t. chi, e, B", "dtype": "f32",
                   "forward_ms": f_ms, "adjoint_ms": a_ms, "ratio": a_ms / f_ms,
                   "adjoint_updates_per_s": nupd / (a_ms * 1e-3), "reps": args.adjoint_reps,
                   "launch": ctx.adjoint_info(),
                   "timing": "CUDA events inside porta_emergent_vjp (forward emergent sweep with tape; "
                             "adjoint sweep + fixed-order reduction), median"}

    # gradients through Jacobi iterations (same box and emergent rays): forward
    # iterations keeping rho checkpoints, then the checkpointed reverse pass
    iter_adj = None
    if args.iter_adjoint != "0" and wl.name == "pol64":
        niter, ckpt = (int(x) for x in args.iter_adjoint.split(","))
        mu, az = synth.emergent_directions()
        nz, ny, nx = ctx.shape
        gen = torch.Generator(device=dev).manual_seed(4321)
        gout = torch.randn((len(mu), ctx.nnu, ny, nx, ctx.ns), dtype=torch.float64, device=dev, generator=gen)
        gbuf = [torch.empty((nz, ny, nx), dtype=torch.float64, device=dev) for _ in range(2)]
        gbuf.append(torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            ctx.set_adjoint_launch(args.adjoint_cluster, args.adjoint_nu_group)
            # warm-up: one iteration and its reverse (times the launch shapes once)
            ctx.set_rho(wl.rho0)
            ctx.iterate_ckpt(1, 1, residual=False)
            ctx.iterate_vjp(mu, az, gout, g_chi=gbuf[0], g_f=gbuf[1], g_b=gbuf[2])
            ctx.set_rho(wl.rho0)
            barrier()
            ev[0].record(stream)
            ctx.iterate_ckpt(niter, ckpt, residual=False)
            ev[1].record(stream)
            ctx.iterate_vjp(mu, az, gout, g_chi=gbuf[0], g_f=gbuf[1], g_b=gbuf[2])
            ev[2].record(stream)
            barrier()
        fwd_ms, rev_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        iter_adj = {"workload": f"{nx}x{ny}x{nz} polarized, {ctx.nnu} frequencies, {ctx.nray} rays, "
                                f"{niter} Jacobi iterations, checkpoints every {ckpt}; loss on the vertical + "
                                "4 oblique emergent rays; gradients w.r.t. chi, f = eps B, B", "dtype": "f32 sweeps, f64 SEE",
                    "forward_ms": fwd_ms, "reverse_ms": rev_ms, "ratio": rev_ms / fwd_ms,
                    "launch": ctx.adjoint_info(), "phases": ctx.iterate_timing(),
                    "timing": "CUDA events around porta_iterate_ckpt (eager iterations + checkpoint copies) "
                              "and porta_iterate_vjp (recomputation, SEE and formal-solution adjoints)"}

    # non-linear multigrid on the same box: 3 levels (64^3 -> 32^3 -> 16^3), V-cycles of
    # 2 pre- and 4 post-smoothing Jacobi iterations and 8 on the coarsest grid, from
    # rho0; Jacobi iterations of the same fine-grid cost (7 sweeps per cycle) beside it
    mgres = None
    if args.mg_cycles > 0 and wl.name == "pol64":
        with torch.cuda.stream(stream):
            ctx.mg_setup(3)
            ctx.set_rho(wl.rho0)
            ctx.mg_vcycle(2, 4, 8)                          # warm-up
            ctx.set_rho(wl.rho0)
            barrier()
            cyc = []
            for _ in range(args.mg_cycles):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ch = ctx.mg_vcycle(2, 4, 8)
                e1.record(stream)
                e1.synchronize()
                cyc.append((e0.elapsed_time(e1), ch))
            ctx.set_rho(wl.rho0)
            jac = []
            for _ in range(args.mg_cycles):
                jac.append(ctx.run_iterations(7))
        mgres = {"levels": ctx.mg_levels(), "cycle": "2 pre + 4 post Jacobi, 8 on the coarsest, from S00 = B",
                 "vcycle_ms": [round(t, 3) for t, _ in cyc], "vcycle_max_change": [c for _, c in cyc],
                 "jacobi_ms_per_7_iterations": 7 * step_ms,
                 "jacobi_max_change_after_7k_iterations": jac,
                 "note": "max_change: of the whole V-cycle for MG, of the last iteration for Jacobi"}

    # multilevel atom without polarization: five levels, four lines, 31 frequencies per
    # line, 160 rays on the 128 x 128 x 96 grid; one Jacobi iteration (formal solution
    # of every line in one batched launch, sums, FP64 rate equations) per step
    mlres = None
    if args.ml_steps > 0 and wl.name == "pol64":
        nxm, nym, nzm = (int(v) for v in args.ml_grid.split(","))
        atm_ml = synth.multilevel_box(nxm, nym, nzm, seed=rank)
        atom = synth.multilevel_atom(seed=rank)
        g = 2.0 * atom["J"] + 1
        pops0 = g * np.exp(-atom["E"] / atm_ml["kT"][..., None])
        pops0 /= pops0.sum(-1, keepdims=True)                  # LTE start
        mctx = P.MlContext(atm_ml, atom, N_MU, N_CHI, 31, precision=P.PORTA_FP32)
        mctx.set_stream(stream)
        mctx.set_atmosphere(atm_ml)
        mctx.set_pops(pops0)
        with torch.cuda.stream(stream):
            mctx.autotune()
            mctx.set_pops(pops0)
            mctx.run_iterations(1, residual=False)              # warm-up (graph capture)
            barrier()
            evm = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.ml_steps)]
            chg = []
            for k in range(args.ml_steps):
                flush.zero_()
                evm[k][0].record(stream)
                mctx.run_iterations(1, residual=False)
                evm[k][1].record(stream)
            barrier()
            chg = mctx.ml_iterate(1)
            # non-linear multigrid on 128x128x96 -> 64x64x48 -> 32x32x24 from LTE
            mctx.mg_setup(3)
            mctx.set_pops(pops0)
            mg_cyc = []
            for _ in range(args.ml_mg_cycles):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ch = mctx.mg_vcycle(2, 4, 8)
                e1.record(stream)
                e1.synchronize()
                mg_cyc.append((e0.elapsed_time(e1), ch))
            mctx.set_pops(pops0)
            jac_ch = [mctx.ml_iterate(7) for _ in range(args.ml_mg_cycles)]
        ml_ms = sum(e[0].elapsed_time(e[1]) for e in evm) / args.ml_steps
        nupd = len(atom["A"]) * 31 * NRAY * nxm * nym * nzm
        mlres = {"workload": f"{nxm}x{nym}x{nzm}, five-level atom (J = 0,1,2,1,2), four lines x 31 frequencies, "
                             f"{NRAY} rays, populations only (FP32 sweeps, FP64 rate equations)",
                 "ms_per_iteration": ml_ms, "updates_per_iteration": nupd,
                 "updates_per_s": nupd / (ml_ms * 1e-3), "steps": args.ml_steps,
                 "max_change_after": chg, "launch": mctx.launch_info(),
                 "multigrid": {"levels": mctx.mg_levels(), "cycle": "2 pre + 4 post Jacobi, 8 on the coarsest, from LTE",
                               "vcycle_ms": [round(t, 1) for t, _ in mg_cyc],
                               "vcycle_max_change": [c for _, c in mg_cyc],
                               "jacobi_max_change_after_7k_iterations": jac_ch},
                 "timing": "CUDA events around one graph replay per step, L2 flushed between steps"}
        mctx.close()

    # polarized multilevel atom (all rho^K_Q of the five levels, 69 per voxel) on the
    # same grid and quadratures: FP32 sweeps of the four lines (polarized formal
    # solver), FP64 rate equations one warp per voxel
    mlpol = None
    if args.mlpol_steps > 0 and wl.name == "pol64":
        nxm, nym, nzm = (int(v) for v in args.ml_grid.split(","))
        atm_ml = synth.multilevel_box(nxm, nym, nzm, seed=rank)
        atom = synth.multilevel_atom(seed=rank)
        g = 2.0 * atom["J"] + 1
        pops0 = g * np.exp(-atom["E"] / atm_ml["kT"][..., None])
        pops0 /= pops0.sum(-1, keepdims=True)
        # Zeeman splitting per gauss small enough for the first-order term at the
        # field tails of this atmosphere (2 zeta |B|max (x_max + |v|max) < 1)
        pctx = P.MlContext(atm_ml, atom, N_MU, N_CHI, 31, precision=P.PORTA_FP32, polarized=True, zeta=ML_ZETA)
        pctx.set_stream(stream)
        pctx.set_atmosphere(atm_ml)
        pctx.set_pops(pops0)
        with torch.cuda.stream(stream):
            pctx.autotune()
            pctx.set_pops(pops0)
            pctx.run_iterations(1, residual=False)              # warm-up (graph capture)
            barrier()
            evp = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.mlpol_steps)]
            for k in range(args.mlpol_steps):
                flush.zero_()
                evp[k][0].record(stream)
                pctx.run_iterations(1, residual=False)
                evp[k][1].record(stream)
            barrier()
            # the formal solutions and sums alone (eager), for the split
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            pctx.ml_formal_solve(want=False)
            e1.record(stream)
            barrier()
            pch = pctx.ml_iterate(1)
            # multigrid V-cycle of the polarized atom (3 levels) from LTE
            pmg = []
            if args.mlpol_mg_cycles > 0:
                pctx.mg_setup(3)
                pctx.set_pops(pops0)
                for _ in range(args.mlpol_mg_cycles):
                    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e2.record(stream)
                    chm = pctx.mg_vcycle(2, 4, 8)
                    e3.record(stream)
                    e3.synchronize()
                    pmg.append((e2.elapsed_time(e3), chm))
        p_ms = sum(e[0].elapsed_time(e[1]) for e in evp) / args.mlpol_steps
        fs_ms = e0.elapsed_time(e1)
        nupd = len(atom["A"]) * 31 * NRAY * nxm * nym * nzm
        mlpol = {"workload": f"{nxm}x{nym}x{nzm}, five-level atom (J = 0,1,2,1,2), all rho^K_Q (69 per voxel), "
                             f"zeta = {ML_ZETA} per G, "
                             f"four lines x 31 frequencies, {NRAY} rays (FP32 sweeps of the polarized formal solver, "
                             "FP64 rate equations)",
                 "ms_per_iteration": p_ms, "formal_solution_ms": fs_ms, "rate_equations_ms": p_ms - fs_ms,
                 "updates_per_iteration": nupd, "updates_per_s": nupd / (p_ms * 1e-3),
                 "steps": args.mlpol_steps, "max_change_after": pch, "launch": pctx.launch_info(),
                 "multigrid": {"levels": pctx.mg_levels(), "cycle": "2 pre + 4 post Jacobi, 8 on the coarsest, from LTE",
                               "vcycle_ms": [round(t, 1) for t, _ in pmg],
                               "vcycle_max_change": [c for _, c in pmg]} if pmg else None,
                 "timing": "CUDA events around one graph replay per step (L2 flushed); formal_solution_ms: one eager "
                           "formal solution + sums; rate_equations_ms: the difference"}
        pctx.close()

    # max over ranks
    if world > 1:
        step_ms, sweep_ms, e2e_s = max_over_ranks([step_ms, sweep_ms, e2e_s], dev)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    achieved = F_ALG * wl.updates / (sweep_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, sample = wl.oracle_sample(args.cpu_sample_rays)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    cfg = {"workload": wl.desc, **wl.config, "updates_per_step": wl.updates, "seed": "rank",
           "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}",
           "sweep_launch": info, "sweep_fill": fill, "launch_shape": "forced" if forced else "autotuned",
           "step": "one CUDA-graph replay of a Jacobi iteration (sweep, J^K_Q sums, SEE, residual)"}
    line = {
        "metric": METRIC, "value": job_throughput(wl.updates, world, step_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / PEAK_FP32_TFLOPS,
                     "traffic": measured_traffic() if wl.name == "pol64" else None,
                     "kernel": "sweep_kernel<float,4,JKQ>", "flops_per_update": F_ALG,
                     "kernel_ms": sweep_ms,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived, not measured)"},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": job_throughput(wl.updates, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "residual": residual},
        "gpu_launches": (4 if fill["cluster"] > 0 else 3) * args.steps,
        "fp64_plain": fp64,
        "adjoint": adjoint,
        "multigrid": mgres,
        "iter_adjoint": iter_adj,
        "multilevel": mlres,
        "multilevel_polarized": mlpol,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = args_parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
