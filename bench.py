"""Benchmark of the UGKWP-LTS steady-iteration step on B300.

Workload (N = 1): hypersonic flow past a cylinder in the dense regime, Kn = 0.01 (freestream mean free path
over the diameter), Ma = 15, T_w = T_inf, body-fitted O-mesh 240 radial x 320 circumferential, first layer
1e-4 D, outer boundary at 20 D, N_ref = 150 particles per cell, CFL 0.8, local time stepping, production
precision (FP32 particles, 64-bit fixed-point tallies, FP64 cell update): the largest single-GPU
configuration. The state is first advanced from the uniform freestream through its start-up transient (a
peak near 1e8 particles) until the particle count settles (changes by less than 1% over 1,000 steps, checked
every 500 steps; about 5.3e6 particles); then W warm-up steps and K timed steps. One step is one full pass of
the method over the domain.

Timing: every timed step is bracketed by CUDA events on the library's stream, and an L2 flush (a 512 MB
write) precedes each step outside the events. value = particle-steps / summed step time. The dominant
kernel (particle transport and tallies) is timed by the library's own stage events over a profiled window
that follows the timed steps (same state, eager launches, every stage on the library's stream).

With N = 1 the line also carries `convergence`: steps and wall-clock to a 1e-6 residual (particle-free
mode, all FP64) and to a steady drag and heat load (stochastic method), LTS against GTS, on the 120 x 160
cylinder at Kn 0.1, Ma 5 (the dense cylinder reaches no 1e-6 within minutes); `--no-convergence` skips it.

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
import tempfile
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


def bench_case(args=None):
    """The throughput workload: the dense-regime Kn 0.01 cylinder (the default), with --case kn01 the Kn 0.1 one, with
    --case tri the cylinder at Kn 0.1 on the radius on the hybrid unstructured mesh of the paper's cell count,
    with --case tri_kn001 / tri_plate the stand-ins of the paper's other two unstructured meshes."""
    which = getattr(args, "case", "kn001") if args is not None else "kn001"
    if which == "kn001":
        return wl.case_cylinder_kn001()
    if which == "tri":
        return wl.case_cylinder_tri()
    if which == "tri_kn001":
        return wl.case_cylinder_tri_kn001()
    if which == "tri_plate":
        return wl.case_plate_tri()
    return wl.case_cylinder_kn01()


WORKLOADS = {
    "cylinder_120x160_Kn0.1_Ma5.0": "cylinder O-mesh 120x160, Kn=0.1 (lambda/D), Ma=5, Tw/Tinf=1, N_ref=100, CFL 0.8, LTS",
    "cylinder_240x320_Kn0.01_Ma15.0": "cylinder O-mesh 240x320, Kn=0.01 (lambda/D), Ma=15, Tw/Tinf=1, N_ref=150, CFL 0.8, LTS",
    "cylinder_tri_7420_Kn0.05_Ma5.0": "cylinder hybrid unstructured mesh, 7420 cells (1820 quadrilaterals in 13 wall "
                                      "layers, 5600 triangles), wall cell 0.01 R, Kn=0.05 (lambda/D; 0.1 on R), Ma=5, "
                                      "Tw/Tinf=1, N_ref=100, CFL 0.8, LTS",
    "cylinder_tri_16100_Kn0.005_Ma5.0": "cylinder hybrid unstructured mesh, 16100 cells (2100 quadrilaterals in 15 wall "
                                        "layers, 14000 triangles), wall cell 0.0005 R, Kn=0.005 (lambda/D; 0.01 on R), "
                                        "Ma=5, Tw/Tinf=1, N_ref=100, CFL 0.8, LTS",
    "plate_tri_5885_Kn0.0169_Ma20.2": "flat plate hybrid unstructured mesh, 5885 cells (1605 quadrilaterals in 15 wall "
                                      "rows, 4280 triangles), first cell 1e-5 L, Kn=0.0169 (lambda/L), Ma=20.2, "
                                      "Tw/Tinf=290/13.32, Maxwell wall alpha=0.85, monatomic, N_ref=200, CFL 0.8, LTS",
}


def config_dict(case, burn, flush):
    return {"workload": WORKLOADS.get(case.name, case.name),
            "cells": case.mesh.ncells, "mode": "LTS", "precision": "FP32 particles, int64 fixed-point tallies, "
            "FP64 cell update", "burn_in_steps": burn, "l2": flush, "parallelism": "replicas (one case per GPU)"}


def burn_in(solver, args):
    """Advance the fresh state through its start-up transient: a fixed number of steps (--burn >= 0), or until
    the particle count changes by less than 1% over 1,000 steps (checked every 500 steps, at least 5,000
    steps, at most --burn-max)."""
    if args.burn >= 0:
        solver.step(args.burn)
        return args.burn, f"fixed: {args.burn} steps"
    hist = []
    steps = 0
    while steps < args.burn_max:
        solver.step(500)
        steps += 500
        hist.append(solver.num_particles())
        if steps >= 5000 and len(hist) >= 3 and abs(hist[-1] - hist[-3]) < 0.01 * hist[-1]:
            break
    return steps, ("until the particle count changed by less than 1% over 1,000 steps (checked every 500, "
                   f"at least 5,000, at most {args.burn_max}); counts at the last checks {hist[-3:]}")


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
    case = bench_case(args)
    # the product's recommended mode: one captured graph per step, launch shape chosen by the autotuner
    # the dense-regime cylinder overshoots its steady particle count in the start-up transient (about 9 N_ref per
    # cell, 1.03e8 particles near step 1,500, against 5.3e6 once settled)
    cap = 12 * case.n_ref * case.mesh.ncells if args.case in ("kn001", "tri_kn001") else 0
    if args.capacity:
        cap = args.capacity
    solver = ugkwp.Solver(case, precision=0, seed=rank, stream=stream.cuda_stream, use_graph=True, order=args.order,
                          capacity=cap)
    if args.load_state:
        # a burned-in state saved by an earlier run of this workload (--save-state): the profiling runs start
        # from it, so that the profiled process launches few kernels before the captured ones
        solver.load_checkpoint(args.load_state)
        burn, burn_rule = int(solver.stats()[0]), f"loaded from a checkpoint of a burned-in run ({args.load_state})"
    else:
        burn, burn_rule = burn_in(solver, args)
        if args.save_state:
            solver.save(args.save_state)
    if args.launch:
        solver.set_launch(*[int(v) for v in args.launch.split(",")])
    launch, tune_ms = solver.autotune(16) if not args.no_autotune else (solver.launch(), None)
    stream.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.fill_(1.0)
        solver.step(1)
    torch.cuda.synchronize()
    s0 = solver.stats()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local, os.path.join(tempfile.gettempdir(), f"ugkwp_clocks_rank{rank}_{os.getpid()}.csv")) \
        if rank == 0 else None
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
    s1 = solver.stats()
    psteps = int(s1[8] - s0[8])
    ncells_steps = case.mesh.ncells * args.steps
    ms_all, ps_all = reduce_over_ranks(ms, float(psteps), world, "cuda")
    # per-stage device times (events around each stage on the stream that runs it; eager launches) over a
    # separate profiled window of the same run: the stage breakdown and the transport kernel's duration
    nprof_steps = min(args.steps, args.profile_steps)
    solver.set_profiling(True)
    solver.profile()
    p0 = solver.stats()
    for k in range(nprof_steps):
        flush.fill_(float(k))
        solver.step(1)
    stage_ms, nprof = solver.profile()
    solver.set_profiling(False)
    p1 = solver.stats()
    prof_psteps = int(p1[8] - p0[8])
    e2e = run_e2e(args, solver, stream) if rank == 0 and not args.no_e2e else None
    if rank == 0:
        peaks, which = _peaks()
        part_ms = stage_ms["particles"] / max(nprof, 1)
        per_launch = prof_psteps / max(nprof, 1)
        achieved = BYTES_PER_PARTICLE_STEP * per_launch / (part_ms * 1e-3) / 1e9
        traffic = particles_traffic(per_launch, case.name)
        cpu = cpu_baseline(args, solver) if not args.no_cpu_baseline else None
        cfg = config_dict(case, burn, "512 MB L2 flush before every timed step, outside the events")
        cfg["burn_in_rule"] = burn_rule
        cfg["reconstruction_order"] = args.order
        kname = {1: "k_particles (warp-chunked)",
                 2: f"k_particles_warp + k_particles_fly ({launch[0]}-particle warp tiles, bulk async copies, "
                    f"{launch[1]} CTAs/SM, records updated in place; crossing particles in a flight pass)"}
        cfg["launch"] = {"transport_kernel": kname[launch[3]],
                         "chunk": launch[0], "blocks_per_sm": launch[1],
                         "sort_every": launch[2],
                         "chosen_by": "autotuner" if not args.no_autotune else
                         ("--launch" if args.launch else "defaults"), "graph": True}
        line = {
            "metric": "particle-steps/s", "value": ps_all / (ms_all * 1e-3), "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded; uniform freestream start)",
            "config": cfg,
            "cell_updates_per_s": world * ncells_steps / (ms_all * 1e-3),
            "particles_per_step": psteps / args.steps,
            "stage_ms_per_step": {k: v / max(nprof, 1) for k, v in stage_ms.items()},
            "stage_window": f"{nprof} further steps, eager launches with per-stage events, every stage on the "
                            "library's stream (the second stream's ghost sources and wave fluxes not overlapped)",
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                         "kernel": {1: "k_particles", 2: "k_particles_warp + k_particles_fly"}[launch[3]] +
                                   " (t_f draw, transport with dt_R/dt_L scaling, tallies, compaction)",
                         "algorithmic_bytes_per_launch": BYTES_PER_PARTICLE_STEP * per_launch,
                         "peak_source": f"{which} (MEASURED_PEAKS.json hbm_gbs)"},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": ck,
            "gpu_launches": gpu_launches_per_step(case, args.order) * args.steps,
            "wall_s_timed": t_wall,
            "last_step": {"particles": int(s1[1]), "new": int(s1[2]), "collided_removed": int(s1[3]),
                          "left_domain": int(s1[4]), "face_crossings": int(s1[5]), "wall_hits": int(s1[6])},
        }
    solver.close()
    if rank == 0:
        if world == 1 and not args.no_convergence:
            line["convergence"] = convergence_summary(args, stream)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def transport_source_hash(t) -> str:
    """16 hex digits of the SHA-256 of the transport kernel's source: the region of the core unit between the
    two markers recorded in the traffic file (the per-cell views, the fixed-point helpers, the sampling, the
    free flight and k_particles) followed by the deterministic-math header it includes."""
    import hashlib
    txt = open(os.path.join(ROOT, t["source"]), encoding="utf-8").read()
    a, b = txt.index(t["region_start"]), txt.index(t["region_end"])
    h = hashlib.sha256(txt[a:b].encode())
    for extra in t.get("extra_sources", []):
        h.update(open(os.path.join(ROOT, extra), "rb").read())
    return h.hexdigest()[:16]


def particles_traffic(per_launch: float, workload: str):
    """DRAM bytes (read + written) of one transport-kernel launch: the bytes per particle of the committed ncu
    capture (profiles/particles_traffic.json) times this launch's particles; None when the transport kernel's
    source has changed since the capture or the workload is not the captured one."""
    tfile = os.path.join(ROOT, "profiles", "particles_traffic.json")
    try:
        t = json.load(open(tfile))
        if transport_source_hash(t) != t["region_sha256_16"] or t["workload"] != workload:
            return None
        return float(t["bytes_per_particle"]) * per_launch
    except (OSError, KeyError, ValueError):
        return None


def reduce_over_ranks(ms: float, work: float, world: int, device: str):
    """Job time = max over ranks of the timed milliseconds; job work = sum over ranks (independent replicas,
    no data-path collective: this is the only cross-rank communication)."""
    if world <= 1:
        return ms, work
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0])


def gpu_launches_per_step(case, order=1):
    # begin-step, decompose, 3 scan kernels, sample, particles, the wave fluxes (first order, production: the
    # per-cell FP32 preparation, the wall-cell faces when the mesh has walls, the FP32 faces and the FP64
    # retry; order 2: the gradients and one FP64 kernel), 3 scan kernels and the scatter (they return at once
    # except on sort steps), update; the ghost-source parameter and particle kernels when the mesh has
    # far-field or fixed faces; the heat-flux tally when Pr != 1
    m = case.mesh
    if hasattr(m, "cells"):
        tags = list(m.boundary[:, 2])
    else:
        tags = list(m.bc_imin) + list(m.bc_imax) + list(m.bc_jmin) + list(m.bc_jmax)
    ghosts = any(t in (wl.BC_FARFIELD, wl.BC_FIXED) for t in tags)
    walls = any(t == wl.BC_WALL for t in tags)
    flux = 2 if order == 2 else 3 + (1 if walls else 0)
    # the warp-staged transport is two kernels (stay pass, flight pass)
    return 12 + flux + (2 if ghosts else 0) + (1 if case.Pr != 1.0 else 0)


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


def cpu_baseline(args, solver=None):
    """The oracle (plain C, one thread) on a bounded sample of the same workload: the device's burned-in state
    (cell field, retained tally, particles) loaded into the oracle (for timing only), then full steps for
    about --cpu-seconds."""
    from oracle import binding as ob
    case = bench_case(args)
    o = ob.Oracle(case, precision=0)
    if solver is not None:
        W, _ = solver.field()
        o.set_state(int(solver.stats()[0]), W, solver.tallies()["wret"], solver.particles())
        what = "the device's burned-in state loaded into the oracle (timing only)"
    else:
        o.step(1)
        what = "the freestream start (after 1 untimed step)"
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
            "sample": f"{steps} full steps ({n0 / max(steps, 1):.3g} particles per step) of the same workload from "
                      f"{what}"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import binding as ob
    case = bench_case(args)
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


def run_convergence(args):
    """Steps and wall-clock to convergence, LTS vs GTS, on the chosen workload (--case)."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    print(json.dumps(converge_case(bench_case(args), args, stream)))


def convergence_summary(args, stream):
    """The convergence comparison of the bench line: the 120 x 160 cylinder at Kn 0.1, Ma 5 (LTS against GTS)."""
    out = converge_case(wl.case_cylinder_kn01(), args, stream, verbose=False)
    out["note"] = ("residual: raw / freestream scale (ugkwp_residual); steady: EMA (alpha 2/1001) of drag and "
                   "heat load (device monitors, ugkwp_monitors) within max(1%, 3 sigma) of the final-window mean; "
                   "wall clock includes a monitor read-back every step (both modes); warm start: bench.py --mode "
                   "warmstart")
    return out


def converge_case(case, args, stream, verbose=True):
    """(i) the deterministic particle-free mode (GKS limit, all FP64) to a 1e-6 residual (the library's
    freestream-normalised residual), with the steps at which 1e-3 .. 1e-6 were crossed; (ii) the full
    stochastic method (production precision) to "steady": the EMA (alpha = 2/1001) of the drag and heat-load
    coefficients stays within the tolerance of its final-window mean."""
    from paper_2607_09552_b300 import steady, ugkwp
    out = {"mode": "convergence", "workload": config_dict(case, 0, "n/a")["workload"],
           "reconstruction_order": args.order, "results": {}}
    for ts in ("LTS", "GTS"):
        gts = ts == "GTS"
        r = {}
        out["results"][ts] = r
        if not args.skip_wave:
            s = ugkwp.Solver(case, gts=gts, precision=1, wave_only=True, stream=stream.cuda_stream, use_graph=True,
                             order=args.order)
            w = steady.run_to_residual(s, 1e-6, args.max_wave_steps, 500)
            r["wave_only_fp64"] = {"steps_to_1e-6": w["steps"] if w["converged"] else None,
                                   "wall_s": w["seconds"], "final_residual": w["residual"],
                                   "ms_per_step": 1e3 * w["seconds"] / w["steps"],
                                   "marks": {f"{k:.0e}": v for k, v in w["marks"].items()}}
            s.close()
            if verbose:
                print(json.dumps({"phase": f"{ts} wave_only", **r}), flush=True)
        if args.skip_stochastic:
            continue
        n = args.lts_steps if not gts else args.gts_steps
        # GTS keeps far more particles (every cell samples with the smallest time step): larger capacity
        cap = (32 if gts else 8) * case.n_ref * case.mesh.ncells
        s = ugkwp.Solver(case, gts=gts, precision=0, stream=stream.cuda_stream, use_graph=True, capacity=cap,
                         order=args.order)
        hcd, hch, hp, hq, hres, hnp, ht = [], [], [], [], [], [], []
        t0 = time.perf_counter()
        try:
            for k in range(n):
                s.step(1)
                mon = s.monitors()   # the device's monitored loads (C_d, C_H, stagnation C_p, C_Q)
                hcd.append(mon[0])
                hch.append(mon[1])
                hp.append(mon[2])
                hq.append(mon[3])
                ht.append(time.perf_counter() - t0)
                if k % 100 == 0:
                    hres.append(float(np.max(s.residual()[:4])))
                    hnp.append(s.num_particles())
        except ugkwp.UgkwpError as e:
            r["stochastic_error"] = f"step {len(hcd)}: {e}; particles {hnp[-3:]}"
            if verbose:
                print(json.dumps({"phase": f"{ts} stochastic", **r}), flush=True)
            s.close()
            continue
        kd, _ = steady.steady_step(hcd)
        kh, _ = steady.steady_step(hch)
        k_st = max(kd, kh)
        tail = slice(int(0.8 * n), n)
        r["stochastic"] = {"steps_run": n, "steps_to_steady": k_st if k_st < n else None,
                           "wall_s_to_steady": ht[k_st - 1] if 0 < k_st < n else None, "wall_s_run": ht[-1],
                           "ms_per_step": 1e3 * ht[-1] / n, "steady_drag_step": kd, "steady_heat_step": kh,
                           "Cd": float(np.mean(hcd[tail])), "CH": float(np.mean(hch[tail])),
                           "stagnation_Cp": float(np.mean(hp[tail])),
                           "stagnation_CQ": float(np.mean(hq[tail])),
                           "residual_plateau": float(np.median(hres[len(hres) // 2:])),
                           "particles_mean": float(np.mean(hnp[len(hnp) // 2:])), "particles_max": int(np.max(hnp)),
                           }
        if verbose:
            r["stochastic"]["drag_history_every_500"] = [round(x, 5) for x in hcd[::500]]
        s.close()
        if verbose:
            print(json.dumps({"phase": f"{ts} stochastic", **r}), flush=True)
    L, G = out["results"]["LTS"], out["results"]["GTS"]
    lw, gw = L.get("wave_only_fp64", {}), G.get("wave_only_fp64", {})
    if lw.get("steps_to_1e-6") and gw.get("steps_to_1e-6"):
        out["wave_only_speedup_steps"] = gw["steps_to_1e-6"] / lw["steps_to_1e-6"]
        out["wave_only_speedup_wall"] = gw["wall_s"] / lw["wall_s"]
    ls, gs = L.get("stochastic", {}), G.get("stochastic", {})
    if ls.get("steps_to_steady") and gs.get("steps_to_steady"):
        out["stochastic_speedup_steps"] = gs["steps_to_steady"] / ls["steps_to_steady"]
        out["stochastic_speedup_wall"] = gs["wall_s_to_steady"] / ls["wall_s_to_steady"]
    return out


def run_batch(args):
    """The seeded 16-case sweep (cylinders and plates, Kn, Ma, T_w drawn from seed 0) advanced together: one
    graph of per-case streams per step, the batched persistent kernel (4 and 6 CTAs per SM), and the same cases
    stepped one after another (each with its own graph); same states throughout (the cases continue from one
    timing to the next)."""
    import torch
    from paper_2607_09552_b300 import ugkwp
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = wl.batch_sweep(0, scale=args.batch_scale)
    # room for the start-up transient, whose particle count overshoots the steady one (up to about 9 N_ref per cell)
    solvers = [ugkwp.Solver(c, precision=0, stream=stream.cuda_stream, use_graph=True,
                            capacity=12 * c.n_ref * c.mesh.ncells) for c in cases]
    for s in solvers:
        s.step(args.burn if args.burn >= 0 else 3000)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(run):
        """(particle-steps/s, ms per step) of args.steps steps after args.warmup untimed ones"""
        run(args.warmup)
        torch.cuda.synchronize()
        p0 = sum(int(s.stats()[8]) for s in solvers)
        e0.record(stream)
        run(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        p1 = sum(int(s.stats()[8]) for s in solvers)
        return (p1 - p0) / (ms * 1e-3), ms / args.steps

    def sequential(n):
        for _ in range(n):
            for s in solvers:
                s.step(1)

    out = {"mode": "batch", "steps": args.steps, "warmup": args.warmup}
    b = ugkwp.Batch(solvers, stream=stream.cuda_stream)
    out["graph_particle_steps_per_s"], out["graph_ms_per_step"] = timed(b.step)
    b.close()
    for cps in (4, 6):
        b = ugkwp.Batch(solvers, stream=stream.cuda_stream, persistent=True, ctas_per_sm=cps)
        plan = b.plan()
        out[f"persistent{cps}_particle_steps_per_s"], out[f"persistent{cps}_ms_per_step"] = timed(b.step)
        st = b.status()
        b.close()
        if st[0] != 0:
            raise RuntimeError(f"persistent batch stopped: {st}")
        out[f"persistent{cps}_plan"] = {"items_per_step": plan[1], "ctas": plan[2], "ctas_per_sm": plan[3]}
    out["sequential_particle_steps_per_s"], out["sequential_ms_per_step"] = timed(sequential)
    out["cases"] = [{"name": c.name, "cells": c.mesh.ncells, "Kn": c.Kn, "Ma": c.Ma, "Tw": c.Tw, "n_ref": c.n_ref,
                     "particles": s.num_particles()} for c, s in zip(cases, solvers)]
    print(json.dumps(out))


def _eval_wave(e, c, ref, fam, nets, args, st):
    """Particle-free FP64 solve of one held-out case from the freestream and from the network."""
    import torch
    from paper_2607_09552_b300 import steady, ugkwp
    from paper_2607_09552_b300 import warmstart as ws
    s = ugkwp.Solver(c, precision=1, wave_only=True, stream=st, use_graph=True)
    rc = steady.run_to_residual(s, 1e-6, args.eval_wave_max, 500, ref)
    W_cold = s.field()[0]
    s.close()
    t0 = time.perf_counter()
    s = ugkwp.Solver(c, precision=1, wave_only=True, stream=st, use_graph=True)
    s.warm_start(nets[fam], ws.FAMILY_MAPS[fam])
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    rw = steady.run_to_residual(s, 1e-6, args.eval_wave_max, 500, ref)
    W_warm = s.field()[0]
    s.close()
    e["wave_only_fp64"] = {"cold_steps": rc["steps"] if rc["converged"] else None, "cold_s": rc["seconds"],
                           "warm_steps": rw["steps"] if rw["converged"] else None,
                           "warm_s": rw["seconds"] + t_inf, "warm_start_s": t_inf,
                           "cold_final": rc["residual"], "warm_final": rw["residual"],
                           "cold_marks": {f"{k:.0e}": v for k, v in rc["marks"].items()},
                           "warm_marks": {f"{k:.0e}": v for k, v in rw["marks"].items()},
                           "state_rel_diff": float(np.max(np.abs(W_warm - W_cold)) / np.max(np.abs(W_cold)))}


def _eval_stoch(c, warm, net, fam, n, navg, st):
    """Stochastic LTS run of one held-out case (production precision) from the freestream or the network:
    steps and seconds to steady (drag and heat-load EMA), final-window loads, surfaces averaged over the
    last navg steps."""
    from paper_2607_09552_b300 import steady, ugkwp
    from paper_2607_09552_b300 import warmstart as ws
    s = ugkwp.Solver(c, precision=0, stream=st, use_graph=True)
    if warm:
        s.warm_start(net, ws.FAMILY_MAPS[fam])
    hcd, hch, ht = [], [], []
    t0 = time.perf_counter()
    for k in range(n):
        s.step(1)
        if k == n - navg:
            s.reset_surface()
        mon = s.monitors()
        hcd.append(mon[0])
        hch.append(mon[1])
        ht.append(time.perf_counter() - t0)
    kd, _ = steady.steady_step(hcd)
    kh, _ = steady.steady_step(hch)
    k_st = max(kd, kh)
    r = {"steps_to_steady": k_st if k_st < n - navg else None,
         "wall_s_to_steady": ht[k_st - 1] if 0 < k_st < n - navg else None,
         "Cd": float(np.mean(hcd[-navg:])), "CH": float(np.mean(hch[-navg:])), "surface": s.surface(averaged=True)}
    s.close()
    return r


def scaled_residual(case, solver):
    """Largest raw residual component in freestream units: sqrt(sum_i Omega_i (dW/dt)^2) divided by
    (rho U, rho U^2, rho U^2, rho U^3 / 2) / L times the square root of the domain area, so that an O(1)
    flux imbalance over the whole domain reads about 1 whatever the first step looked like."""
    r = solver.residual()[4:]
    U = wl.freestream_speed(case.Ma)
    area = float(np.sum(solver.geometry()[1]))
    scale = np.array([U, U * U, U * U, 0.5 * U ** 3]) * np.sqrt(area)
    return float(np.max(r / scale))


def run_warmstart(args):
    """Learned warm start (all on the GPU): converged particle-free fields of seeded sweeps of 16 uneven
    cases (cylinders and plates, batched graph launches) train one network per geometry family; then held-out
    seeded cases are solved from the freestream and from the network: (i) particle-free, all FP64, to a 1e-6
    residual (relative to the freestream start's first step), each case alone and, warm-started, all cases in
    one batched launch; (ii) the stochastic method to steady (drag and heat-load EMA), with the averaged wall
    p, tau_w, q of the warm-started run against the freestream-started one."""
    import torch
    from paper_2607_09552_b300 import steady, ugkwp
    from paper_2607_09552_b300 import warmstart as ws
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    out = {"mode": "warmstart", "train": {}, "eval": []}
    sets = {"cylinder": ws.TrainingSet(), "plate": ws.TrainingSet()}
    t_all = time.perf_counter()
    for seed in range(args.train_sweeps):
        cases = wl.batch_sweep(seed)
        solvers = [ugkwp.Solver(c, precision=0, wave_only=True, stream=st) for c in cases]
        b = ugkwp.Batch(solvers, stream=st)
        t0, steps = time.perf_counter(), 0
        res = [1.0] * len(solvers)
        failed = {}
        while steps < args.train_max_steps:
            b.step(1000)
            steps += 1000
            for i, (c, sv) in enumerate(zip(cases, solvers)):
                if i in failed:
                    continue
                try:
                    res[i] = scaled_residual(c, sv)
                except ugkwp.UgkwpError as e:
                    failed[i] = str(e)
                    res[i] = 0.0
            if max(res) < args.train_tol:
                break
        used = 0
        for i, (c, sv) in enumerate(zip(cases, solvers)):
            # a field still far from steady (or one that failed) would teach the network a transient
            if i not in failed and res[i] < args.train_accept:
                sets[ws.family(c)].add(sv, ws.FAMILY_MAPS[ws.family(c)])
                used += 1
        b.close()
        for sv in solvers:
            sv.close()
        out["train"][f"sweep{seed}"] = {"steps": steps, "seconds": time.perf_counter() - t0,
                                        "max_residual": max(res), "median_residual": float(np.median(res)),
                                        "failed": {cases[i].name: m for i, m in failed.items()}, "fields_used": used,
                                        "residuals": {c.name: r for c, r in zip(cases, res)}}
        print(json.dumps({"phase": f"training fields, sweep {seed}", **out["train"][f"sweep{seed}"]}), flush=True)
    nets = {}
    for fam, tset in sets.items():
        if not tset.sizes:
            out["train"][fam] = {"fields": 0, "note": "no converged training field: this family starts cold"}
            continue
        feats, targs = tset.tensors()
        net = ws.new_network(0)
        t0 = time.perf_counter()
        hist = ws.train(net, feats, targs, steps=args.train_steps, batch=8192, lr=2e-3, log_every=args.train_steps // 4)
        torch.cuda.synchronize()
        nets[fam] = net
        out["train"][fam] = {"rows": int(feats.shape[0]), "fields": len(tset.sizes), "adam_steps": args.train_steps,
                             "seconds": time.perf_counter() - t0, "loss": hist}
        print(json.dumps({"phase": f"train {fam}", **out["train"][fam]}), flush=True)
        del feats, targs
    out["train"]["total_seconds"] = time.perf_counter() - t_all
    # held-out cases
    cases = []
    for geo, kn, ma, tw in wl.held_out_conditions(1000, args.eval_cyl, args.eval_plate):
        if geo == "cylinder":
            c = wl.case_cylinder(120, 160, 1e-3, 15.0, Kn=kn, Ma=ma, Tw=tw, n_ref=100)
        else:
            c = wl.case_plate(Kn=kn, Ma=ma, Tw=tw, n_ref=50)
        cases.append(c)
    refs = [steady.first_residual(c, precision=1, wave_only=True, stream=st) for c in cases]
    # (i) particle-free FP64 to 1e-6: cold alone, warm alone, warm batched
    cold_total = warm_total = 0.0
    for c, ref in zip(cases, refs):
        fam = ws.family(c)
        e = {"case": c.name, "family": fam, "Kn": c.Kn, "Ma": c.Ma, "Tw": c.Tw}
        out["eval"].append(e)
        if fam not in nets:
            e["wave_only_fp64"] = {"note": "no network for this family"}
            continue
        try:
            _eval_wave(e, c, ref, fam, nets, args, st)
        except ugkwp.UgkwpError as err:
            e["wave_only_fp64"] = {"error": str(err)}
            print(json.dumps({"phase": "eval wave-only", **e}), flush=True)
            continue
        cold_total += e["wave_only_fp64"]["cold_s"]
        warm_total += e["wave_only_fp64"]["warm_s"]
        print(json.dumps({"phase": "eval wave-only", **e}), flush=True)
    t0 = time.perf_counter()
    solvers = []
    for c in cases:
        s = ugkwp.Solver(c, precision=1, wave_only=True, stream=st)
        if ws.family(c) in nets:
            s.warm_start(nets[ws.family(c)], ws.FAMILY_MAPS[ws.family(c)])
        solvers.append(s)
    b = ugkwp.Batch(solvers, stream=st)
    done, steps = [None] * len(solvers), 0
    while steps < args.eval_wave_max and any(d is None for d in done):
        b.step(500)
        steps += 500
        for i, (s, ref) in enumerate(zip(solvers, refs)):
            if done[i] is None:
                try:
                    if float(np.max(s.residual()[4:] / ref)) < 1e-6:
                        done[i] = steps
                except ugkwp.UgkwpError as err:
                    done[i] = f"error: {err}"
    batched_s = time.perf_counter() - t0
    b.close()
    for s in solvers:
        s.close()
    out["wave_only_fp64_totals"] = {"cold_sequential_s": cold_total, "warm_sequential_s": warm_total,
                                    "warm_batched_s": batched_s, "warm_batched_steps": done,
                                    "speedup_warm_batched_vs_cold": cold_total / batched_s}
    print(json.dumps({"phase": "eval wave-only totals", **out["wave_only_fp64_totals"]}), flush=True)
    # (ii) stochastic method to steady: cold vs warm, averaged surfaces after steady
    n, navg = args.eval_stoch_steps, 1000
    for e, c in zip(out["eval"], cases):
        fam = ws.family(c)
        res = {}
        for start in ("cold", "warm"):
            if start == "warm" and fam not in nets:
                res[start] = {"note": "no network for this family"}
                continue
            try:
                res[start] = _eval_stoch(c, start == "warm", nets.get(fam), fam, n, navg, st)
            except ugkwp.UgkwpError as err:
                res[start] = {"error": str(err)}
        if "surface" in res["cold"] and "surface" in res["warm"]:
            pc, tc, qc = res["cold"].pop("surface")
            pw, tw_, qw = res["warm"].pop("surface")
            res["surface_rel_err"] = {"p": float(np.linalg.norm(pw - pc) / np.linalg.norm(pc)),
                                      "tau_w": float(np.linalg.norm(tw_ - tc) / (np.sqrt(len(tc)) * np.max(np.abs(tc)))),
                                      "q": float(np.linalg.norm(qw - qc) / np.linalg.norm(qc))}
        for r_ in res.values():
            r_.pop("surface", None)
        e["stochastic"] = res
        print(json.dumps({"phase": "eval stochastic", "case": c.name, **res}), flush=True)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--burn", type=int, default=-1,
                    help="burn-in steps; -1: until the particle count changes by < 1%% over 1,000 steps")
    ap.add_argument("--burn-max", type=int, default=40000)
    ap.add_argument("--no-convergence", action="store_true")
    ap.add_argument("--capacity", type=int, default=0, help="particle capacity (0: the workload's default)")
    ap.add_argument("--save-state", default="", help="save the burned-in state (checkpoint) to this file")
    ap.add_argument("--load-state", default="", help="start from a saved burned-in state instead of burning in")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch", default="", help="chunk,blocks_per_sm,sort_every,transport set before the "
                    "(optional) autotuning pass; with --no-autotune the launch shape that is timed")
    ap.add_argument("--profile-steps", type=int, default=400)
    ap.add_argument("--mode", default="throughput", choices=["throughput", "convergence", "batch", "warmstart"])
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--case", default="kn001", choices=["kn01", "kn001", "tri", "tri_kn001", "tri_plate"])
    ap.add_argument("--order", type=int, default=1, choices=[1, 2],
                    help="reconstruction order of the wave fluxes (2: second order, FP64 wave fluxes)")
    ap.add_argument("--max-wave-steps", type=int, default=400000)
    ap.add_argument("--lts-steps", type=int, default=30000)
    ap.add_argument("--gts-steps", type=int, default=150000)
    ap.add_argument("--skip-wave", action="store_true")
    ap.add_argument("--skip-stochastic", action="store_true",
                    help="convergence mode: the particle-free FP64 runs only (the dense cylinder's GTS stochastic "
                         "run outgrows any capacity)")
    ap.add_argument("--train-sweeps", type=int, default=4)
    ap.add_argument("--train-tol", type=float, default=1e-5)
    ap.add_argument("--train-max-steps", type=int, default=60000)
    ap.add_argument("--train-steps", type=int, default=60000)
    ap.add_argument("--train-accept", type=float, default=1e-3)
    ap.add_argument("--eval-cyl", type=int, default=4)
    ap.add_argument("--eval-plate", type=int, default=4)
    ap.add_argument("--eval-wave-max", type=int, default=200000)
    ap.add_argument("--eval-stoch-steps", type=int, default=20000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "convergence":
        run_convergence(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "warmstart":
        run_warmstart(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
