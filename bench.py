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
UPDATES = NX * NY * NZ * NRAY * N_NU
WORKLOAD = ("polarized two-level atom (Jl=0->Ju=1, Hanle + weak-field Zeeman), random box 64x64x64, "
            "160 rays, 21 frequencies; one Jacobi iteration per step (FP32 sweeps, FP64 SEE)")
# algorithmic floating-point operations per voxel.ray.frequency update of the
# formal solution (stage-by-stage count of the method, each node's transfer
# coefficients counted once per ray and frequency; derivation in the design doc)
F_ALG = 293
# FP32 issue peak of the GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz
SMS, LANES, SM_MAX_MHZ = 152, 128, 2070.0
PEAK_FP32_TFLOPS = SMS * LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
L2_FLUSH_BYTES = 256 << 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "sweep_pol64_traffic.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1307_4217_gb300", "csrc", f)
                  for f in ("sweep.cu", "device_math.cuh", "porta_internal.cuh")]


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
    ap.add_argument("--cluster", type=int, default=0, help="force the sweep cluster size (skips the autotuner)")
    ap.add_argument("--nu-group", type=int, default=0, help="force frequencies per pass (skips the autotuner)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


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

    # Each rank solves its own box (independent replicas: weak scaling, no data-path collective).
    atm = synth.random_box(NX, NY, NZ, seed=rank)
    rho0 = np.zeros((NZ, NY, NX, 6))
    rho0[..., 0] = atm["bpl"]
    stream = torch.cuda.Stream(device=dev)

    forced = args.cluster > 0 or args.nu_group > 0

    def make(precision):
        ctx = P.Context(atm, P.PORTA_MODEL_TWOLEVEL_HANLE, N_MU, N_CHI, N_NU, precision=precision,
                        cluster=args.cluster, nu_group=args.nu_group)
        ctx.set_stream(stream)
        ctx.set_atmosphere(atm)
        ctx.set_rho(rho0)
        if not forced:
            ctx.autotune()          # launch-shape autotuner (outside the timed region)
            ctx.set_rho(rho0)
        return ctx

    ctx = make(P.PORTA_FP32)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.formal_solve()
            ctx.accumulate_jkq(want=False)
            ctx.see_update(residual=False)
        barrier()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        sampler = ClockSampler(local)
        sampler.start()
        barrier()
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (outside the events)
            ev[k][0].record(stream)
            ctx.formal_solve()
            ev[k][1].record(stream)
            ctx.accumulate_jkq(want=False)
            ctx.see_update(residual=False)
            ev[k][2].record(stream)
        barrier()
        clocks = sampler.stop()
    step_ms = sum(e[0].elapsed_time(e[2]) for e in ev) / args.steps
    sweep_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    info = ctx.launch_info()
    residual = None

    # end to end through the ABI with pinned host buffers: rho in, J^K_Q + Lambda* + residual out
    rho_h = torch.from_numpy(rho0.copy()).pin_memory()
    jkq_h = torch.empty((NZ, NY, NX, 6), dtype=torch.float64).pin_memory()
    ls_h = torch.empty((NZ, NY, NX), dtype=torch.float64).pin_memory()
    with torch.cuda.stream(stream):
        for _ in range(1):
            ctx.set_rho(rho_h)
            ctx.formal_solve()
            ctx.accumulate_jkq(jkq_h, ls_h)
            ctx.see_update()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_rho(rho_h)
            ctx.formal_solve()
            ctx.accumulate_jkq(jkq_h, ls_h)
            residual = ctx.see_update()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = rho_h.numel() * 8
    d2h = (jkq_h.numel() + ls_h.numel() + 1) * 8

    # FP64 plain form of the same step
    fp64 = None
    if args.fp64_steps > 0:
        ctx64 = make(P.PORTA_FP64)
        with torch.cuda.stream(stream):
            ctx64.formal_solve()
            ctx64.accumulate_jkq(want=False)
            ctx64.see_update(residual=False)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.fp64_steps):
                ctx64.formal_solve()
                ctx64.accumulate_jkq(want=False)
                ctx64.see_update(residual=False)
            e1.record(stream)
            barrier()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        fp64 = {"value": world * UPDATES / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "dtype": "f64",
                "launch": ctx64.launch_info()}
        ctx64.close()

    # max over ranks
    if world > 1:
        t = torch.tensor([step_ms, sweep_ms, e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms, sweep_ms, e2e_s = t.tolist()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    achieved = F_ALG * UPDATES / (sweep_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, dt, sample = oracle_sample(args.cpu_sample_rays)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    line = {
        "metric": METRIC, "value": world * UPDATES / (step_ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "rays": NRAY, "frequencies": N_NU,
                   "updates_per_step": UPDATES, "seed": "rank", "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{world}", "sweep_launch": info,
                   "launch_shape": "forced" if forced else "autotuned"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / PEAK_FP32_TFLOPS, "traffic": measured_traffic(),
                     "kernel": "sweep_kernel<float,4,JKQ>", "flops_per_update": F_ALG,
                     "kernel_ms": sweep_ms,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived, not measured)"},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "e2e": {"value": world * UPDATES / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "residual": residual},
        "gpu_launches": 3 * args.steps,
        "fp64_plain": fp64,
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
