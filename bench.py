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
# FP32 issue peak of the GB300 from its unit counts (152 SMs x 128 FP32 lanes x 2
# flops per FMA x 2070 MHz); the roofline uses the measured peak (porta_fma_peak)
SMS, LANES, SM_MAX_MHZ = 152, 128, 2070.0
PEAK_FP32_TFLOPS_NOMINAL = SMS * LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_pol64_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1307_4217_gb300", "csrc", f)
                  for f in ("sweep_j.cu", "sweep_common.cuh", "device_math.cuh", "porta_internal.cuh")]


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
    ap.add_argument("--batch-steps", type=int, default=3,
                    help="timed Jacobi iterations of the 256-box batch beside the default workload (0 skips them)")
    ap.add_argument("--c0", type=int, default=1, help="time the unpolarized 16x16x32 box to convergence (0 skips it)")
    ap.add_argument("--faces", type=int, default=1,
                    help="time the formal solution with short characteristics on the first cell face (0 skips it)")
    ap.add_argument("--faces-grid", type=int, default=64,
                    help="box of that section, n^3 (64: the benchmark box; a smaller one for profiling captures)")
    ap.add_argument("--solver-family", type=int, default=1,
                    help="E(dtau) of the Sec. 3.4 solver family on the sigmoid benchmark (0 skips it)")
    ap.add_argument("--peak-seconds", type=float, default=1.0, help="device time per FMA-peak measurement")
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
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def wait_first(self, timeout=5.0):
        """Block until the sampler has written its first row (nvidia-smi takes a few
        hundred ms to start), so that the timed region that follows is sampled."""
        t_end = time.time() + timeout
        while self.proc is not None and time.time() < t_end and self.proc.poll() is None:
            with open(self.path) as f:
                if "\n" in f.read():
                    return
            time.sleep(0.02)

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

def _oracle_ray(args):
    import oracle
    atm, m = args
    p = oracle.Problem(atm, oracle.MODEL_HANLE, N_MU, N_CHI, N_NU)
    oracle.formal_solve(p, oracle.initial_rho(p, atm), rays_range=(m, m + 1))
    return m


def oracle_sample_all_cores(seed=0):
    """Time the FP64 oracle, as it stands, on all host cores: one full ray (all 21
    frequencies, the whole 64^3 box) per core, rays spread over the hemispheres,
    in a process pool (spawned: the GPU context of this process is not shared)."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    atm = synth.random_box(NX, NY, NZ, seed=seed)
    rays = np.linspace(0, NRAY - 1, ncores).astype(int)
    with mp.get_context("spawn").Pool(ncores) as pool:
        pool.map(_oracle_ray, [(atm, int(rays[0]))] * min(ncores, 2))   # start-up (imports, library load)
        t0 = time.perf_counter()
        pool.map(_oracle_ray, [(atm, int(m)) for m in rays], chunksize=1)
        dt = time.perf_counter() - t0
    n = ncores * NX * NY * NZ * N_NU
    return n / dt, dt, ncores, (f"{ncores} rays x 21 frequencies over the full 64^3 box, one ray per core "
                                f"({n} updates, {dt:.1f} s)")


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
    from paper_1307_4217_gb300 import shard

    # measured FMA peaks of this GPU (the roofline's denominator): FP32 FFMA and
    # packed FFMA2 chains (the better of the two is the FP32 peak), FP64 DFMA
    peaks = {}
    for kind, name in ((0, "fp32_ffma"), (1, "fp32_ffma2"), (2, "fp64_dfma")):
        rc, tf, ms = P.porta_fma_peak(kind, args.peak_seconds if kind < 2 else 0.5 * args.peak_seconds)
        peaks[name] = tf if rc == P.PORTA_OK else None
    peak_fp32 = max(v for k, v in peaks.items() if k.startswith("fp32") and v) if any(peaks.values()) else None

    # N > 1: the ranks split the frequencies of every formal solution of the same box
    # (bands, one all-reduce of the partial sums per iteration: strong scaling); N = 1:
    # one context, one captured Jacobi iteration per step
    wl = Workload(args.workload, 0 if world > 1 else rank)
    bands = world > 1
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
    if bands:
        band_it = shard.BandIteration(ctx, rank, world, device=dev)
        ctx.autotune()                      # the band's own launch shape
        ctx.set_rho(wl.rho0)

        def step(residual=False):
            return band_it.step(residual=residual)
    else:
        band_it = None

        def step(residual=False):
            return ctx.run_iterations(1, residual=residual)
    swept = wl.updates if not bands else wl.updates * (band_it.band[1] - band_it.band[0]) // N_NU

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        # warm-up: eager calls, then the captured graph of one Jacobi iteration
        for _ in range(args.warmup):
            if bands:
                step()
            else:
                ctx.formal_solve()
                ctx.accumulate_jkq(want=False)
                ctx.see_update(residual=False)
        step()
        barrier()
        # timed steps: one graph replay (formal solution, J^K_Q sums, SEE, residual) each;
        # with bands: the band's formal solution, one all-reduce of the partial sums, the update
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
        sampler = ClockSampler(local)
        sampler.start()
        sampler.wait_first()
        barrier()
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            step()
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
        step(residual=True)
        ctx.get_rho(rho_out)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_rho(rho_h)
            residual = step(residual=True)
            ctx.get_rho(rho_out)
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = rho_h.numel() * 8
    d2h = rho_out.numel() * 8 + 8

    # FP64 plain form of the same step (single box only: the FP64 batch takes ~15 s per step)
    fp64 = None
    accuracy = None
    if args.fp64_steps > 0 and wl.name == "pol64" and world == 1:
        ctx64 = make(P.PORTA_FP64)
        with torch.cuda.stream(stream):
            ctx64.run_iterations(1, residual=False)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx64.run_iterations(args.fp64_steps, residual=False)
            e1.record(stream)
            barrier()
            # accuracy of the FP32 form against the FP64 form (which the parity tests hold to
            # 1e-10 of the FP64 oracle) on the benchmarked box: one formal solution and one
            # update from the same unknowns, in the benchmarked launch shape
            out = {}
            for name, cc in (("f32", ctx), ("f64", ctx64)):
                cc.set_rho(wl.rho0)
                cc.formal_solve()
                jj, ll = cc.accumulate_jkq()
                cc.see_update(residual=False)
                out[name] = (jj, ll, cc.get_rho())
            barrier()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        fp64 = {"value": world * wl.updates / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "dtype": "f64",
                "launch": ctx64.launch_info()}
        (j32, l32, r32), (j64, l64, r64) = out["f32"], out["f64"]
        s = np.abs(j64[..., :1])
        accuracy = {
            "against": "the FP64 form on the same box (parity-tested to 1e-10 of the FP64 oracle)",
            "J00_rel": float(np.max(np.abs(j32[..., 0] - j64[..., 0]) / s[..., 0])),
            "J2Q_abs_over_J00": float(np.max(np.abs(j32[..., 1:] - j64[..., 1:]) / s)),
            "lambda_rel": float(np.max(np.abs(l32 - l64) / np.abs(l64))),
            "S00_rel_after_update": float(np.max(np.abs(r32[..., 0] - r64[..., 0]) / np.abs(r64[..., 0]))),
            "sigma2Q_abs_after_update": float(np.max(np.abs(r32[..., 1:] / r32[..., :1] - r64[..., 1:] / r64[..., :1]))),
            "tolerance": "1e-5 relative on J00 and Lambda*, 1e-5 J00 on J2Q",
        }
        ctx64.close()

    # reverse mode of the emergent Stokes profiles (differentiation workload: the
    # same 64^3 box, vertical + 4 oblique emergent rays, all frequencies), FP32:
    # device time of the forward sweep with its tape and of the adjoint sweep
    adjoint = None
    if args.adjoint_reps > 0 and wl.name == "pol64" and world == 1:
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
            # the forward emergent formal solution alone (no tape), same directions
            eout = torch.empty((len(mu), ctx.nnu, ny, nx, ctx.ns), dtype=torch.float64, device=dev)
            ctx.emergent_stokes(mu, az, out=eout)                                     # shape tuning
            tf = []
            for _ in range(args.adjoint_reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.emergent_stokes(mu, az, out=eout)
                e1.record(stream)
                e1.synchronize()
                tf.append(e0.elapsed_time(e1))
        f_ms = float(np.median([t["forward_ms"] for t in ts]))
        a_ms = float(np.median([t["adjoint_ms"] for t in ts]))
        f0_ms = float(np.median(tf))
        nupd = len(mu) * ctx.nnu * nx * ny * nz
        adjoint = {"workload": f"{nx}x{ny}x{nz} polarized, {ctx.nnu} frequencies, vertical + 4 oblique (mu=0.5) "
                               "emergent rays; gradients w.r.t. chi, e, B", "dtype": "f32",
                   "forward_ms": f_ms, "adjoint_ms": a_ms, "ratio": a_ms / f_ms,
                   "forward_notape_ms": f0_ms, "ratio_vs_forward_notape": a_ms / f0_ms,
                   "adjoint_updates_per_s": nupd / (a_ms * 1e-3), "reps": args.adjoint_reps,
                   "launch": ctx.adjoint_info(),
                   "timing": "CUDA events inside porta_emergent_vjp (forward emergent sweep with tape; "
                             "adjoint sweep + fixed-order reduction), median; forward_notape_ms: CUDA events "
                             "around porta_emergent_stokes of the same directions (no tape), median"}

    # gradients through Jacobi iterations (same box and emergent rays): forward
    # iterations keeping rho checkpoints, then the checkpointed reverse pass
    iter_adj = None
    if args.iter_adjoint != "0" and wl.name == "pol64" and world == 1:
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
    if args.mg_cycles > 0 and wl.name == "pol64" and world == 1:
        with torch.cuda.stream(stream):
            ctx.mg_setup(3)
            ctx.set_rho(wl.rho0)
            ctx.mg_vcycle(2, 4, 8)                          # warm-up
            ctx.set_rho(wl.rho0)
            barrier()
            cyc = []
            res0 = ctx.residual()
            for _ in range(args.mg_cycles):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ch = ctx.mg_vcycle(2, 4, 8)
                e1.record(stream)
                e1.synchronize()
                cyc.append((e0.elapsed_time(e1), ch, ctx.residual()))
            # the tri-cubic-centered prolongation, and the nested method (Sec. 5.1: the
            # coarsest grid's problem first, each finer level from the prolonged solution)
            ctx.mg_set_prolongation(3)
            ctx.set_rho(wl.rho0)
            cub = []
            for _ in range(args.mg_cycles):
                ctx.mg_vcycle(2, 4, 8)
                cub.append(ctx.residual())
            ctx.set_rho(wl.rho0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.mg_nested(1, 2, 4, 8)
            e1.record(stream)
            e1.synchronize()
            nested = {"ms": e0.elapsed_time(e1), "residual": [ctx.residual()]}
            for _ in range(args.mg_cycles - 1):
                ctx.mg_vcycle(2, 4, 8)
                nested["residual"].append(ctx.residual())
            ctx.mg_set_prolongation(1)
            ctx.set_rho(wl.rho0)
            jac, jres = [], []
            for _ in range(args.mg_cycles):
                jac.append(ctx.run_iterations(7))
                jres.append(ctx.residual())
        mgres = {"levels": ctx.mg_levels(), "cycle": "2 pre + 4 post Jacobi, 8 on the coarsest, from S00 = B",
                 "vcycle_cubic_residual": cub,
                 "nested": dict(nested, note="one nested pass (8 Jacobi on 16^3, then 1 V-cycle on 32^3 and on 64^3, "
                                             "tri-cubic prolongation), then tri-cubic V-cycles; residual after each"),
                 "vcycle_ms": [round(t, 3) for t, _, _ in cyc], "vcycle_max_change": [c for _, c, _ in cyc],
                 "residual_start": res0, "vcycle_residual": [r for _, _, r in cyc],
                 "jacobi_ms_per_7_iterations": 7 * step_ms,
                 "jacobi_max_change_after_7k_iterations": jac, "jacobi_residual_after_7k_iterations": jres,
                 "note": ("max_change: of the whole V-cycle for MG, of the last iteration for Jacobi; residual: "
                          "porta_residual, max over voxels of |f - A(x)| relative to the voxel's largest unknown; "
                          "7 Jacobi iterations cost the fine-grid formal solutions of one V-cycle (2 + 4 + 1)")}

    # multilevel atom without polarization: five levels, four lines, 31 frequencies per
    # line, 160 rays on the 128 x 128 x 96 grid; one Jacobi iteration (formal solution
    # of every line in one batched launch, sums, FP64 rate equations) per step
    mlres = None
    if args.ml_steps > 0 and wl.name == "pol64" and world == 1:
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
            ml_res0 = mctx.residual()
            for _ in range(args.ml_mg_cycles):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ch = mctx.mg_vcycle(2, 4, 8)
                e1.record(stream)
                e1.synchronize()
                mg_cyc.append((e0.elapsed_time(e1), ch, mctx.residual()))
            mctx.set_pops(pops0)
            jac_ch, jac_res = [], []
            for _ in range(args.ml_mg_cycles):
                jac_ch.append(mctx.ml_iterate(7))
                jac_res.append(mctx.residual())
        ml_ms = sum(e[0].elapsed_time(e[1]) for e in evm) / args.ml_steps
        nupd = len(atom["A"]) * 31 * NRAY * nxm * nym * nzm
        mlres = {"workload": f"{nxm}x{nym}x{nzm}, five-level atom (J = 0,1,2,1,2), four lines x 31 frequencies, "
                             f"{NRAY} rays, populations only (FP32 sweeps, FP64 rate equations)",
                 "ms_per_iteration": ml_ms, "updates_per_iteration": nupd,
                 "updates_per_s": nupd / (ml_ms * 1e-3), "steps": args.ml_steps,
                 "max_change_after": chg, "launch": mctx.launch_info(),
                 "multigrid": {"levels": mctx.mg_levels(), "cycle": "2 pre + 4 post Jacobi, 8 on the coarsest, from LTE",
                               "vcycle_ms": [round(t, 1) for t, _, _ in mg_cyc],
                               "vcycle_max_change": [c for _, c, _ in mg_cyc],
                               "residual_start": ml_res0, "vcycle_residual": [r for _, _, r in mg_cyc],
                               "jacobi_max_change_after_7k_iterations": jac_ch,
                               "jacobi_residual_after_7k_iterations": jac_res},
                 "timing": "CUDA events around one graph replay per step, L2 flushed between steps"}
        mctx.close()

    # polarized multilevel atom (all rho^K_Q of the five levels, 69 per voxel) on the
    # same grid and quadratures: FP32 sweeps of the four lines (polarized formal
    # solver), FP64 rate equations one warp per voxel
    mlpol = None
    if args.mlpol_steps > 0 and wl.name == "pol64" and world == 1:
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
                    pmg.append((e2.elapsed_time(e3), chm, pctx.residual()))
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
                               "vcycle_ms": [round(t, 1) for t, _, _ in pmg],
                               "vcycle_max_change": [c for _, c, _ in pmg],
                               "vcycle_residual": [r for _, _, r in pmg]} if pmg else None,
                 "timing": "CUDA events around one graph replay per step (L2 flushed); formal_solution_ms: one eager "
                           "formal solution + sums; rate_equations_ms: the difference"}
        pctx.close()

    # the unpolarized box of 16x16x32 voxels (48 rays, 11 frequencies): Jacobi (ALI)
    # iterations to convergence, FP64 (max relative change < 1e-8) and FP32 (< 1e-6, or its
    # noise floor), graph replays; with no horizontal modulation, the sqrt(eps) law
    c0 = None
    if args.c0 and wl.name == "pol64" and world == 1:
        atm0 = synth.plane_parallel_box(16, 16, 32)
        c0 = {"workload": "unpolarized two-level atom, 16x16x32, eps = 1e-2, B = 1, chi modulated by 1 + 0.2 sin cos, "
                          "48 rays (3 x 8 per hemisphere), 11 frequencies; Jacobi iterations from S = B",
              "updates_per_iteration": 16 * 16 * 32 * 48 * 11}
        for prec, name, tol in ((P.PORTA_FP64, "f64", 1e-8), (P.PORTA_FP32, "f32", 1e-6)):
            cc = P.Context(atm0, P.PORTA_MODEL_TWOLEVEL_UNPOL, 3, 8, 11, precision=prec)
            cc.set_stream(stream)
            cc.set_atmosphere(atm0)
            r0 = np.ones((32, 16, 16, 1))
            cc.set_rho(r0)
            with torch.cuda.stream(stream):
                cc.run_iterations(1, residual=False)             # graph capture (warm-up)
                cc.set_rho(r0)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                n, ch, conv = cc.iterate_to(tol, 2000 if prec == P.PORTA_FP64 else 400, check_every=10)
                e1.record(stream)
                barrier()
            ms = e0.elapsed_time(e1) / n
            c0[name] = {"iterations": n, "last_change": ch, "converged": conv, "tolerance": tol,
                        "ms_per_iteration": ms, "updates_per_s": c0["updates_per_iteration"] / (ms * 1e-3),
                        "timing": "CUDA events around porta_iterate_to (graph replays, change read every 10)"}
            cc.close()
        flat = synth.plane_parallel_box(16, 16, 32, modulation=0.0)
        cc = P.Context(flat, P.PORTA_MODEL_TWOLEVEL_UNPOL, 3, 8, 11, precision=P.PORTA_FP64)
        cc.set_stream(stream)
        cc.set_atmosphere(flat)
        cc.set_rho(np.ones((32, 16, 16, 1)))
        with torch.cuda.stream(stream):
            cc.iterate_to(1e-8, 2000)
        s = cc.get_rho()[..., 0]
        cc.close()
        c0["sqrt_eps_law"] = {"S_top_over_sqrt_eps_B": float(s[-1, 0, 0] / np.sqrt(1e-2)),
                              "column_spread": float(np.max(np.abs(s - s[:, :1, :1])))}

    # the family of formal solvers of Sec. 3.4 on the one-ray sigmoid benchmark (Fig. 5):
    # E(dtau) per method on the GPU (FP64), 200 log-spaced spacings x 4 grid shifts per call
    family = None
    if args.solver_family and wl.name == "pol64" and world == 1:
        names = {P.PORTA_SC_BESSER: "BESSER", P.PORTA_SC_PARABOLIC: "parabolic", P.PORTA_SC_LINEAR: "linear",
                 P.PORTA_SC_BEZIER_FB: "Bezier_FB", P.PORTA_SC_CBEZIER: "CBezier"}
        show = [2.0, 1.0, 0.5, 0.1, 0.01, 0.005]
        family = {"workload": "one ray, constant opacity, S = sigma(2,-5,z) sigma(-2,5,z) on z in [-12, 12], "
                              "exact I at the first node; E = max relative true error (Eq. 18)",
                  "dtau": show, "E": {}}
        dts = np.repeat(np.logspace(np.log10(0.002), np.log10(2.0), 200), 4)
        shifts = dts * np.tile([0.0, 0.25, 0.5, 0.75], 200)
        for m, nm in names.items():
            rc, e_show = P.porta_sigmoid_error(P.PORTA_FP64, m, show)
            t0 = time.perf_counter()
            rc2, e_all = P.porta_sigmoid_error(P.PORTA_FP64, m, dts, shifts)
            dt_call = time.perf_counter() - t0
            family["E"][nm] = [float(x) for x in e_show]
            family.setdefault("call_ms", {})[nm] = dt_call * 1e3
        family["cases_per_call"] = int(dts.size)
        family["timing"] = "wall clock around porta_sigmoid_error (host copies and one launch, one thread per case)"

    # the same formal solution with M and P on the first cell face crossed (vertical faces for
    # grazing rays: each such plane solved by ordered line sweeps repeated to convergence)
    faces = None
    if args.faces and wl.name == "pol64" and world == 1:
        fctx, f_updates, f_desc = ctx, wl.updates, wl.desc.split(";")[0]
        if args.faces_grid != 64:
            # a smaller box of the same statistics (profiling captures), S^0_0 = B
            n = args.faces_grid
            fatm = synth.random_box(n, n, n, seed=0)
            fctx = P.Context(fatm, P.PORTA_MODEL_TWOLEVEL_HANLE, *wl.quad, precision=P.PORTA_FP32)
            fctx.set_atmosphere(fatm)
            frho = np.zeros((n, n, n, 6))
            frho[..., 0] = fatm["bpl"]
            fctx.set_rho(frho)
            fctx.set_stream(stream)
            f_updates = n ** 3 * (2 * wl.quad[0] * wl.quad[1]) * wl.quad[2]
            f_desc = f"polarized two-level atom, random box {n}x{n}x{n}, {(2 * wl.quad[0] * wl.quad[1])} rays, {wl.quad[2]} frequencies"
        with torch.cuda.stream(stream):
            fctx.set_sc_faces(0)
            ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            fctx.formal_solve()
            flush.zero_()
            ev0[0].record(stream)
            fctx.formal_solve()
            ev0[1].record(stream)
            jp, lp = fctx.accumulate_jkq()
            p_ms = ev0[0].elapsed_time(ev0[1])
            fctx.set_sc_faces(1)
            fctx.formal_solve()
            jf, lf = fctx.accumulate_jkq()
            evf = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            flush.zero_()
            evf[0].record(stream)
            fctx.formal_solve()
            evf[1].record(stream)
            barrier()
            f_ms = evf[0].elapsed_time(evf[1])
            fctx.set_sc_faces(0)
        if fctx is not ctx:
            fctx.close()
        faces = {"workload": f_desc + "; one J^K_Q formal solution, FP32",
                 "ms": f_ms, "updates_per_s": f_updates / (f_ms * 1e-3),
                 "ratio_to_plane_sweep": f_ms / p_ms,
                 "J00_rel_diff_to_plane_placement": float(np.max(np.abs(jf[..., 0] - jp[..., 0]) / np.abs(jp[..., 0]))),
                 "timing": "CUDA events around one porta_formal_solve with porta_set_sc_faces(1), and one with 0 for the ratio (L2 flushed)"}

    # the 256 boxes of uneven size in one persistent launch per sweep (graph replays)
    batch = None
    if args.batch_steps > 0 and wl.name == "pol64" and world == 1:
        bw = Workload("batched256", rank)
        bc = bw.context(P.PORTA_FP32, args.cluster, args.nu_group)
        bc.set_stream(stream)
        with torch.cuda.stream(stream):
            if not forced:
                bc.autotune()
                bc.set_rho(bw.rho0)
            bc.run_iterations(1, residual=False)
            barrier()
            evb = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.batch_steps)]
            for k in range(args.batch_steps):
                flush.zero_()
                evb[k][0].record(stream)
                bc.run_iterations(1, residual=False)
                evb[k][1].record(stream)
            barrier()
        bms = sum(e[0].elapsed_time(e[1]) for e in evb) / args.batch_steps
        batch = {"workload": bw.desc, "updates_per_iteration": bw.updates, "ms_per_iteration": bms,
                 "updates_per_s": bw.updates / (bms * 1e-3), "launch": bc.launch_info(), "fill": bc.fill_info(),
                 "timing": "CUDA events around one graph replay of a Jacobi iteration, L2 flushed between steps"}
        bc.close()

    # max over ranks
    if world > 1:
        step_ms, sweep_ms, e2e_s = max_over_ranks([step_ms, sweep_ms, e2e_s], dev)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # the sweep's rate over the updates this rank swept (its band, for N > 1)
    achieved = F_ALG * swept / (sweep_ms * 1e-3) / 1e12
    peak = peak_fp32 if peak_fp32 else PEAK_FP32_TFLOPS_NOMINAL
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v1, dt1, sample1 = wl.oracle_sample(args.cpu_sample_rays)
        if wl.name == "pol64":
            v, dt, ncores, sample = oracle_sample_all_cores()
        else:
            v, ncores, sample = v1, 1, sample1
        cpu = {"value": v, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample,
               "single_core": {"value": v1, "cores": 1, "sample": sample1}}
    cfg = {"workload": wl.desc, **wl.config, "updates_per_step": wl.updates, "seed": 0 if world > 1 else "rank",
           "l2": "flushed between timed steps (256 MiB write)",
           "parallelism": (f"frequency bands x{world} (one all-reduce of the int64 partial sums per iteration)"
                           if bands else "one GPU"),
           "sweep_launch": info, "sweep_fill": fill, "launch_shape": "forced" if forced else "autotuned",
           "step": ("the rank's band: formal solution, all-reduce of the partial sums, SEE and residual" if bands else
                    "one CUDA-graph replay of a Jacobi iteration (sweep, J^K_Q sums, SEE, residual)")}
    # kernels per step: sums' set-up, main sweep (+ concurrent filler), sums' finalize, SEE
    per_step = 4 + (1 if fill["cluster"] > 0 else 0)
    line = {
        "metric": METRIC, "value": wl.updates / (step_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "strong" if bands else "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": measured_traffic() if wl.name == "pol64" and not bands else None,
                     "kernel": "jsweep_kernel<float,4>", "flops_per_update": F_ALG,
                     "kernel_ms": sweep_ms, "updates_per_launch": swept,
                     "peak_basis": ("measured: porta_fma_peak, best FP32 FMA chain (FFMA or packed FFMA2) over ~1 s "
                                    "of this GPU" if peak_fp32 else "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (nominal)"),
                     "peaks_measured_tflops": peaks, "peak_nominal_tflops": PEAK_FP32_TFLOPS_NOMINAL},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": wl.updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "residual": residual},
        "gpu_launches": per_step * args.steps,
        "accuracy": accuracy,
        "fp64_plain": fp64,
        "unpolarized_c0": c0,
        "solver_family": family,
        "sc_faces": faces,
        "batched256": batch,
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
