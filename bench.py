"""Benchmark of the UGKWP-LTS steady-iteration step on B300.

Workload (N = 1): hypersonic flow past a cylinder, Kn = 0.1 (freestream mean free path over the diameter),
Ma = 5, T_w = T_inf, body-fitted O-mesh 120 radial x 160 circumferential, first layer 1e-3 D, outer
boundary at 15 D, N_ref = 100 particles per cell (about 1.9 million particles), CFL 0.8, local time
stepping, production precision (FP32 particles, 64-bit fixed-point tallies, FP64 cell update). The state is
first advanced `--burn` steps from the uniform freestream so that the particle population is developed;
then W warm-up steps and K timed steps. One step is one full pass of the method over the domain.

Timing: every timed step is bracketed by CUDA events on the library's stream, and an L2 flush (a 512 MB
write) precedes each step outside the events. value = particle-steps / summed step time. The dominant
kernel (particle transport and tallies) is timed by the library's own stage events over the same steps.

Under torchrun (N > 1) every rank runs an independent replica (seed = rank) of the workload: no data-path
collective, weak scaling; the time is the max over ranks and value the sum of their particle-steps.

`--impl reference` times the CPU oracle (test infrastructure, plain C) on the same workload from the
freestream, one full step per timed step, on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_09552_b300 import workloads as wl  # noqa: E402

BYTES_PER_PARTICLE_STEP = 72.0   # 36-byte particle record (x, y, u, v, w, m: f32; cell: i32; id: u64) read + written


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, idx: int, path: str):
        self.path = path
        self.p = None
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(idx), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken between wall-clock times t0 and t1 (time.time())."""
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        for line in open(self.path):
            t = [x.strip() for x in line.split(",")]
            if len(t) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(t[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if t0 is not None and not (t0 - 0.25 <= ts <= t1 + 0.25):
                    continue
                sm.append(float(t[2]))
                smax.append(float(t[3]))
            except ValueError:
                continue
            for n, v in zip(names, t[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def bench_case():
    return wl.case_cylinder_kn01()


def config_dict(case, burn, flush):
    return {"workload": "cylinder O-mesh 120x160, Kn=0.1 (lambda/D), Ma=5, Tw/Tinf=1, N_ref=100, CFL 0.8, LTS",
            "cells": case.mesh.ncells, "mode": "LTS", "precision": "FP32 particles, int64 fixed-point tallies, "
            "FP64 cell update", "burn_in_steps": burn, "l2": flush, "parallelism": "replicas (one case per GPU)"}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2607_09552_b300 import ugkwp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    case = bench_case()
    solver = ugkwp.Solver(case, precision=0, seed=rank, stream=stream.cuda_stream, use_graph=False)
    solver.step(args.burn)
    stream.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.fill_(1.0)
        solver.step(1)
    torch.cuda.synchronize()
    s0 = solver.stats()
    solver.set_profiling(True)
    solver.profile()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local, os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")) if rank == 0 else None
    time.sleep(0.5)
    t_epoch0 = time.time()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        solver.step(1)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    ck = clocks.stop(t_epoch0, time.time()) if clocks else None
    if world > 1:
        dist.barrier()
    ms = float(sum(a.elapsed_time(b) for a, b in evs))
    stage_ms, nprof = solver.profile()
    solver.set_profiling(False)
    s1 = solver.stats()
    psteps = int(s1[8] - s0[8])
    ncells_steps = case.mesh.ncells * args.steps
    t = torch.tensor([ms, float(psteps)], dtype=torch.float64, device="cuda")
    if world > 1:
        tmax = t.clone()
        dist.all_reduce(tmax[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        ms_all, ps_all = float(tmax[0]), float(t[1])
    else:
        ms_all, ps_all = ms, float(psteps)
    e2e = run_e2e(args, solver, stream) if rank == 0 and not args.no_e2e else None
    if rank == 0:
        peaks, which = _peaks()
        part_ms = stage_ms["particles"] / max(nprof, 1)
        per_launch = psteps / args.steps
        achieved = BYTES_PER_PARTICLE_STEP * per_launch / (part_ms * 1e-3) / 1e9
        traffic = None
        tfile = os.path.join(ROOT, "profiles", "particles_traffic.json")
        if os.path.exists(tfile):
            try:
                traffic = json.load(open(tfile)).get("bytes_per_launch_at_bench_size")
            except Exception:
                traffic = None
        cpu = cpu_baseline(args) if not args.no_cpu_baseline else None
        line = {
            "metric": "particle-steps/s", "value": ps_all / (ms_all * 1e-3), "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; uniform freestream start)",
            "config": config_dict(case, args.burn, "512 MB L2 flush before every timed step, outside the events"),
            "cell_updates_per_s": world * ncells_steps / (ms_all * 1e-3),
            "particles_per_step": per_launch,
            "stage_ms_per_step": {k: v / max(nprof, 1) for k, v in stage_ms.items()},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "kernel": "k_particles (t_f draw, transport with dt_R/dt_L scaling, tallies)",
                         "algorithmic_bytes_per_launch": BYTES_PER_PARTICLE_STEP * per_launch,
                         "peak_source": f"{which} (MEASURED_PEAKS.json hbm_gbs)"},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": ck,
            "gpu_launches": gpu_launches_per_step(case) * args.steps,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line))
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def gpu_launches_per_step(case):
    # decompose, 3 scan kernels, capacity check, sample, particles, wave flux, update, 3 scan kernels,
    # scatter, surface (wall cases), finish
    return 14 + (1 if case.mesh.bc_imin[0] == wl.BC_WALL else 0)


def run_e2e(args, solver, stream):
    """Whole-job pass through the public API from pinned host buffers: upload a full state (cell field,
    retained tally, particles), K steps each followed by a residual read-back, then the field read-back."""
    import torch
    parts = solver.particles()
    W, _ = solver.field()
    wret = solver.tallies()["wret"]
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in parts.items()}
    Wp = torch.from_numpy(W.copy()).pin_memory().numpy()
    wr = torch.from_numpy(wret.copy()).pin_memory().numpy()
    step0 = int(solver.stats()[0])
    torch.cuda.synchronize()
    h2d = Wp.nbytes + wr.nbytes + sum(v.nbytes for v in pin.values())
    s0 = solver.stats()
    t0 = time.perf_counter()
    solver.set_state(step0, Wp, wr, pin)
    out_bytes = 0
    for _ in range(args.steps):
        solver.step(1)
        solver.residual()
        out_bytes += 64
    Wf, _ = solver.field()
    out_bytes += Wf.nbytes * 2
    dt = time.perf_counter() - t0
    s1 = solver.stats()
    return {"value": float(s1[8] - s0[8]) / dt, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d / args.steps,
            "d2h_bytes_per_step": out_bytes / args.steps}


def cpu_baseline(args):
    """The oracle (plain C, one thread) on a bounded sample of the same workload: a few full steps from the
    freestream start."""
    from oracle import binding as ob
    case = bench_case()
    o = ob.Oracle(case, precision=0)
    o.step(1)
    t0 = time.perf_counter()
    n0 = 0
    steps = 0
    while time.perf_counter() - t0 < args.cpu_seconds and steps < 50:
        n_before = o.stats()[1]
        o.step(1)
        n0 += n_before + o.stats()[2]
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": n0 / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} full steps of the same workload from the freestream start (after 1 untimed step)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import binding as ob
    case = bench_case()
    o = ob.Oracle(case, precision=0)
    for _ in range(args.warmup):
        o.step(1)
    psteps = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        n_before = o.stats()[1]
        o.step(1)
        psteps += n_before + o.stats()[2]
    dt = time.perf_counter() - t0
    v = psteps / dt
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; freestream start)",
            "config": config_dict(case, 0, "n/a (CPU)"),
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.warmup} + {args.steps} full steps from the freestream start"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--burn", type=int, default=300)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
