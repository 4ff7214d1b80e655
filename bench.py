#!/usr/bin/env python3
"""Benchmark of the coupled D3Q19 step on the 128 x 128 x 512 settling-sphere
workload (D = 24, density ratio 1.5, Galileo number 144, closed top and bottom).

One benchmark step is one global time step of each coupling variant that
stays stable for a freely settling sphere (PSM M1B1, M2B2: one LBM sweep each;
MEM BB, CLI, MR: two LBM sweeps each, with refilling), each in its own simulation,
FP64 PDFs and arithmetic.  MLUPS counts every lattice cell of every sweep.
(PSM M3B2 runs the same kernel; as printed, with an explicit rigid-body
update, it diverges for a free sphere, so it is not part of the timed step.)

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run: each rank advances its own replicas
(weak scaling, no data-path collective); rank 0 prints the JSON line.
--impl reference times the FP64 CPU oracle (the method as written in the
paper, single node host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline, coupled D3Q19 step; force/velocity error vs FP64"
# k_bulk with FP64 arithmetic is bound by the FP64 pipe (2 FP64 lane-operations
# per SM per cycle on GB300, ncu peak_sustained): its roofline counts FP64
# thread-instructions per cell update, measured by ncu on the 128x128x256
# settling case (DADD + DFMA + DMUL per cell the kernel updates), and the DRAM
# bytes per cell update of the same capture (set to None whenever the kernel
# changes).
K_BULK_F64_DP_INST_PER_CELL = 124.0
K_BULK_F64_DRAM_BYTES_PER_CELL = 292.6
# FP64 operations per cell update as written in the collision (hand count:
# moments 39 -- 18 for rho, 21 for j --, equilibrium base 8, nine pair
# updates 87); the compiler contracts some of them into fused multiply-adds
# (124 issued, above)
K_BULK_F64_DP_OPS_WRITTEN = 134
FP64_LANE_OPS_PER_SM_CLK = 2
COUPLINGS = ("PSM_M1B1", "PSM_M2B2", "MEM_BB", "MEM_CLI", "MEM_MR")
FRAME_COUPLINGS = ("MEM_BB", "MEM_CLI", "MEM_MR", "PSM_M1B1", "PSM_M2B2", "PSM_M3B2")
SHAPE = (128, 128, 512)
WORKLOAD = ("settling sphere 128x128x512, D=24, rho_p/rho_f=1.5, Ga=144 (nu=0.01, tau=0.53), "
            "periodic x/y, no-slip z, released at rest 64 cells below the top; one global step "
            "of each of PSM M1B1/M2B2 (1 sweep) and MEM BB/CLI/MR (2 sweeps, refilling)")
FALLBACK_HBM_GBS = 6800.0


def sweeps_of(coupling: str) -> int:
    return 2 if coupling.startswith("MEM") else 1


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, dist, device) -> float:
    """Largest value over all ranks (the whole-job time); identity without a group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, cells: int, sweeps_per_step: int, steps: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica (weak scaling)."""
    return world * cells * sweeps_per_step * steps / seconds / 1e6


def workload(coupling: str, scale: float):
    from paper_1702_04910_gb300 import workloads as W
    if scale == 1.0:
        return W.settling_sphere(coupling=coupling)
    return W.scaled_settling_sphere(scale, coupling=coupling)


def near_cells(particle, shape, halo=2.0):
    """Cells the near-particle kernel takes: those whose centre lies within
    R + halo of the sphere centre along every axis (host restatement of the
    library's region rule; z is closed)."""
    nx, ny, nz = shape
    R = 0.5 * particle["diameter"]
    count = 1
    for a, (n, periodic) in enumerate(((nx, True), (ny, True), (nz, False))):
        X = particle["x"][a]
        lo = math.ceil(X - R - halo - 0.5)
        hi = math.floor(X + R + halo - 0.5)
        if not periodic:
            lo, hi = max(lo, 0), min(hi, n - 1)
        count *= max(0, min(hi - lo + 1, n))
    return int(count)


def run_ensemble(args, stream, world, dist, barrier, peak, storages=("f64", "f64fx")):
    """The batched ensemble: 64 independent settling cases of uneven size and
    Galileo number advanced by one captured step graph per global step."""
    import numpy as np
    import torch

    from paper_1702_04910_gb300 import workloads as W
    from paper_1702_04910_gb300.binding import Batch

    cases = W.ensemble(args.ensemble_cases, seed=0)
    cells = sum(int(np.prod(c["shape"])) for c in cases)
    # near-particle cell updates per step (MEM cases sweep twice, PSM once)
    near_updates = sum(near_cells(c["particles"][0], c["shape"]) * sweeps_of(c["coupling"])
                       for c in cases)
    out = {}
    for storage in storages:
        b = Batch(cases, storage=storage, stream=stream)
        layouts, grid, tune_ms = b.autotune(reps=3)
        b.profile(True)  # bulk sweeps timed on the device inside the timed steps
        b.step(args.warmup)
        b.synchronize()
        b.profile(True)  # clears the counter: only the timed steps count
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        b.step(args.steps)
        ev1.record()
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        b.synchronize()  # raises if a case reported a device status
        bulk_ms_sum, bulk_sweeps = b.profile_read()
        parts = b.particles()
        cu = b.cell_updates
        # bulk sweeps: every cell update away from the particles, 304 B each,
        # over the device time of the bulk sweeps of a timed step
        bulk_ms = bulk_ms_sum / max(bulk_sweeps, 1)
        sweeps_per_step = bulk_sweeps / max(args.steps, 1)
        bulk_step_ms = bulk_ms_sum / max(args.steps, 1)
        bulk_gbps = 2 * 19 * 8 * (cu - near_updates) / (bulk_step_ms * 1e-3) / 1e9
        out[f"ensemble{len(cases)}_{storage}"] = {
            "value": world * cu * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ms / args.steps, "steps": args.steps, "cases": len(cases),
            "cells": cells, "cell_updates_per_step": cu,
            "workload": "seeded ensemble: D ~ U{8..20}, domain round(5.3D)^2 x round(16D), "
                        "Ga ~ U(100, 250), density ratio 1.5, PSM M1B1/M2B2 and MEM BB/CLI/MR",
            "tuning": {"layouts": {k: layouts.count(k) for k in sorted(set(layouts))},
                       "grid_blocks": grid, "bulk_ms_when_tuned": tune_ms},
            "bulk_avg_launch_ms": bulk_ms, "bulk_sweeps_per_step": sweeps_per_step,
            "bulk_ms_per_step": bulk_step_ms, "bulk_cell_updates_per_step": cu - near_updates,
            "bulk_timing": "device global-timer stamps around every bulk sweep of the "
                           "timed steps (lbm_batch_profile_enable)",
            "bulk_GBps": bulk_gbps, "frac": bulk_gbps / peak,
            "graph_kernels_per_step": b.graph_kernels,
            "gpu_launches": b.graph_kernels * args.steps,
            "device_bytes": b.device_bytes,
            "mean_particle_uz": float(np.mean([p["u"][2] for p in parts])),
            "all_particle_states_finite": bool(all(np.all(np.isfinite(p["u"])) for p in parts)),
        }
        b.close()
    return out


def run_learned(args, stream):
    """Learned force correction: coarse runs corrected towards fine runs of the
    same method; held-out Galileo numbers scored against the plain FP64 fine
    run ("small": D 6 vs 24; "full": D 12 on 64x64x192 in FP32 vs D 48 on
    256x256x768 in FP64)."""
    from paper_1702_04910_gb300 import learned as LR

    full = args.learned == "full"
    # "full" trains on five Galileo numbers (one on each side of both
    # held-out values); "small" on three
    train = [110.0, 130.0, 170.0, 190.0, 240.0] if full else [110.0, 170.0, 240.0]
    res = LR.experiment(train_ga=train, test_ga=[140.0, 210.0],
                        coupling="PSM_M2B2", D_c=12.0 if full else 6.0, ratio=4,
                        t_refs=6.0 if full else 5.0, train_steps=8000 if full else 3000,
                        stream=stream,
                        coarse_storage="f32" if full else "f64")
    res.pop("model").close()
    held = {g: r for g, r in res["cases"].items() if r["held_out"]}
    return {
        "train_ga": res["train_ga"],
        "workload": f"settling sphere Ga {res['test_ga']} held out; coarse D={res['D_coarse']:.0f} "
                    f"({res['coarse_storage']}) corrected towards D={res['D_fine']:.0f} (f64), "
                    f"{res['coupling']}",
        "settling_velocity_rel_error_plain": {g: r["plain"]["mean_rel_error"] for g, r in held.items()},
        "settling_velocity_rel_error_corrected": {g: r["corrected"]["mean_rel_error"] for g, r in held.items()},
        "speedup_vs_fine_fp64": res["speedup_vs_fine_fp64"],
        "training_loss": [res["loss_history"][0], res["loss_history"][-1]],
        "samples": res["samples"], "coarse_steps": res["coarse_steps"],
        "train_steps": res["train_steps"], "train_ms_per_step": res["train_ms_per_step"],
    }


def run_frame_study(args):
    """The paper's benchmark frame (Sec. 4.1) at diameter --frame: case A
    (Ga = 144, compared with Tab. 1) unless --frame-ga / --frame-upv-ref name
    another Galileo number and its reference u_pV."""
    import torch

    from paper_1702_04910_gb300 import frame

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                          "tab1_ga144_upv.txt")
    table = {}
    with open(golden) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                c, d, u = line.split()
                table[(c, int(d))] = float(u)
    out = {}
    for coupling in args.frame_couplings:
        t0 = time.perf_counter()
        r = frame.run_frame(D=args.frame, ga_target=args.frame_ga, u_pv_ref=args.frame_upv_ref,
                            coupling=coupling, storage=args.frame_storage,
                            subcycles=args.frame_subcycles, stream=stream)
        paper = table.get((coupling, int(round(args.frame)))) if args.frame_ga == 144.0 else None
        out[coupling] = {"u_pV": r["u_pV"], "u_pV_paper_tab1": paper,
                         "rel_diff_vs_paper": (abs(r["u_pV"] - paper) / abs(paper)) if paper else None,
                         "Ga": r["calibration"][-1]["Ga"], "nu": r["nu"],
                         "calibration_steps": r["calibration_steps"], "free_steps": r["free_steps"],
                         "seconds": time.perf_counter() - t0}
    print(json.dumps({"frame": f"Ga = {args.frame_ga:g}, reference u_pV {args.frame_upv_ref:g}",
                      "D": args.frame, "storage": args.frame_storage,
                      "shape": frame.frame_shape(args.frame), "results": out}), flush=True)


def run_full_settling(args):
    """The settling workload for its full length: every coupling released at
    rest and run for --full-steps global steps (MEM: two sweeps each) in
    --full-storage, the sphere's height and vertical velocity sampled every
    100 steps, the first step at which it rests on the bottom wall (wall
    contact keeps it one cell off, R13) and where a run became unstable."""
    import numpy as np
    import torch

    from paper_1702_04910_gb300 import workloads as W
    from paper_1702_04910_gb300.binding import LbmError, Simulation
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    for cp in args.couplings:
        case = workload(cp, args.scale)
        s = Simulation(case["shape"], stream=stream, storage=args.full_storage,
                       **W.sim_kwargs(case))
        if args.remap_charge and cp.startswith("MEM"):
            s.set_remap_charge(True)
        s.set_particles(case["particles"])
        s.init_equilibrium()
        R = 0.5 * case["particles"][0]["diameter"]
        samples, contact, failed = [], None, None
        t0 = time.perf_counter()
        done = 0
        while done < args.full_steps:
            n = min(100, args.full_steps - done)
            s.step(n)
            done += n
            try:
                p = s.get_particles()[0]
            except LbmError as e:
                failed = f"{e} (within global steps {done - n}..{done})"
                break
            samples.append([done, round(float(p["x"][2]), 3), round(float(p["u"][2]), 6)])
            if contact is None and p["x"][2] - R <= 1.0 + 1e-9:
                contact = done
        s.close()
        uz = np.array([v[2] for v in samples]) if samples else np.zeros(0)
        out[cp] = {"steps_run": done, "lattice_time": done * sweeps_of(cp), "failed": failed,
                   "wall_contact_step": contact,
                   "max_settling_speed": float(-uz.min()) if uz.size else None,
                   "seconds": time.perf_counter() - t0, "samples_every_100_steps": samples}
    print(json.dumps({"full_settling": WORKLOAD, "steps": args.full_steps,
                      "storage": args.full_storage, "remap_charge": bool(args.remap_charge),
                      "results": out}), flush=True)


def run_lab_drag(args):
    """Drag of a sphere moving relative to the fluid at the same speed in two
    frames: (A) held fixed in the open frame of Sec. 4.1 with a uniform inflow
    from below; (B) translating through fluid at rest in a periodic box
    (density 1e9, so its velocity stays constant).  D = 24, nu = 0.01,
    relative speed 1.24 u_ref of the Ga = 144 case (0.0744).  Both runs use
    two averaged LBM subcycles; the drag is averaged over 50-step windows."""
    import numpy as np
    import torch

    from paper_1702_04910_gb300.binding import Simulation
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    D, nu, U = 24.0, 0.01, 0.0744
    out = {}
    for cp in args.couplings:
        base = dict(coupling=cp, collision="TRT" if cp.startswith("MEM") else "BGK",
                    tau=3.0 * nu + 0.5, magic=3.0 / 16.0, rho0=1.0, subsample=4, subcycles=2,
                    wall_contact=0)
        res = {}
        for frame in ("fixed_in_inflow", "translating_in_fluid_at_rest"):
            if frame == "fixed_in_inflow":
                s = Simulation((128, 128, 384), stream=stream, bc_z=2, inflow=(0.0, 0.0, U),
                               rho_out=1.0, **base)
                s.init_equilibrium(1.0, (0.0, 0.0, U))
                s.set_particles([{"x": (64.0, 64.0, 128.0), "diameter": D, "density": 1.5,
                                  "fixed": 1}])
            else:
                s = Simulation((128, 128, 512), stream=stream, bc_z=0, **base)
                if args.remap_charge and cp.startswith("MEM"):
                    s.set_remap_charge(True)
                s.init_equilibrium(1.0, (0.0, 0.0, 0.0))
                s.set_particles([{"x": (64.0, 64.0, 448.0), "u": (0.0, 0.0, -U), "diameter": D,
                                  "density": 1e9, "fixed": 0}])
            windows = []
            for _ in range(args.lab_drag_windows):
                fz = 0.0
                for _ in range(50):
                    s.step(1)
                    fz += abs(s.forces()[0][0][2])
                windows.append(fz / 50)
            s.close()
            tail = windows[len(windows) // 2:]
            res[frame] = {"drag_second_half_mean": float(np.mean(tail)),
                          "drag_second_half_std": float(np.std(tail)),
                          "drag_windows": [round(v, 5) for v in windows]}
        res["ratio_translating_over_fixed"] = (res["translating_in_fluid_at_rest"]["drag_second_half_mean"]
                                               / res["fixed_in_inflow"]["drag_second_half_mean"])
        out[cp] = res
    print(json.dumps({"lab_drag": "D=24, nu=0.01, relative speed 0.0744 (Ga 144: 1.24 u_ref), "
                                  f"{args.lab_drag_windows} windows of 50 global steps",
                      "remap_charge": bool(args.remap_charge), "results": out}), flush=True)


def run_ensemble_only(args):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    peak, _ = measured_peaks()
    res = run_ensemble(args, stream, 1, None, torch.cuda.synchronize, peak,
                       storages=tuple(args.ensemble_storage.split(",")))
    print(json.dumps(res), flush=True)


def trajectory(case, storage, steps, stream, every=50, profile=False):
    """Release the sphere of `case` and advance it `steps` global steps in
    `storage`; sample the particle's vertical velocity and the vertical
    hydrodynamic force every `every` steps.  Returns (t, u_z, F_z, ms, bulk)
    with ms the CUDA-event time of the run and bulk the mean bulk-sweep
    launch time when profiling."""
    import numpy as np
    import torch

    from paper_1702_04910_gb300 import workloads as W
    from paper_1702_04910_gb300.binding import (LbmError, Simulation, lbm_profile_enable,
                                                lbm_profile_read)
    s = Simulation(case["shape"], stream=stream, storage=storage, **W.sim_kwargs(case))
    s.set_particles(case["particles"])
    s.init_equilibrium()
    lbm_profile_enable(s.h, profile)
    t, uz, fz = [], [], []
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    done = 0
    failed = None
    while done < steps:
        n = min(every, steps - done)
        s.step(n)
        done += n
        try:
            F, _ = s.forces()
            p = s.get_particles()[0]
        except LbmError as e:  # the run became unstable: report where
            failed = f"{e} (within global steps {done - n}..{done})"
            break
        t.append(done)
        uz.append(p["u"][2])
        fz.append(F[0, 2])
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    bulk = None
    if profile and failed is None:
        prof = lbm_profile_read(s.h)
        bulk = prof["bulk"][0] / max(prof["bulk"][1], 1)
    s.close()
    if failed:
        print(f"[bench] {case['coupling']} {storage}: {failed}", file=sys.stderr, flush=True)
    return np.array(t), np.array(uz), np.array(fz), ms, bulk, failed


def settling_errors(make_case, couplings, modes, duration, stream, speed=False, peak=None):
    """Per storage mode: relative error of the settling velocity and of the
    hydrodynamic force against the FP64 run of the same released sphere,
    as means over the last third of `duration` lattice time units after
    release (MEM: duration/2 global steps of two sweeps), plus the largest
    sampled velocity deviation in that window."""
    import numpy as np
    out = {m: {"error_window": f"lattice time {duration - duration // 3}..{duration} after release",
               "settling_velocity_rel_err_vs_f64": {}, "settling_velocity_max_rel_dev_vs_f64": {},
               "force_rel_err_vs_f64": {}} for m in modes}
    info = {}
    esize = {"f64": 8, "f64fx": 8, "f64ff": 8, "f32": 4, "f16s": 2, "bf16s": 2}
    for cp in couplings:
        case = make_case(cp)
        nc = int(np.prod(case["shape"]))
        steps = duration // sweeps_of(cp)
        runs = {m: trajectory(case, m, steps, stream, profile=speed) for m in ["f64"] + list(modes)}
        t, u64, f64_, ms64, _, fail64 = runs["f64"]
        if fail64:
            info[cp] = {"f64_failed": fail64}
            continue
        win = t > steps - steps // 3
        ubar, fbar = u64[win].mean(), f64_[win].mean()
        info[cp] = {"f64_settling_velocity": float(ubar), "f64_force_z": float(fbar),
                    "f64_MLUPS": nc * sweeps_of(cp) * steps / (ms64 * 1e-3) / 1e6}
        for m in modes:
            _, um, fm, msm, bulk, failm = runs[m]
            o = out[m]
            if failm:
                o.setdefault("failed", {})[cp] = failm
                continue
            o["settling_velocity_rel_err_vs_f64"][cp] = float(abs(um[win].mean() - ubar) / abs(ubar))
            o["settling_velocity_max_rel_dev_vs_f64"][cp] = float(np.max(np.abs(um[win] - u64[win])) / abs(ubar))
            o["force_rel_err_vs_f64"][cp] = float(abs(fm[win].mean() - fbar) / abs(fbar))
            if speed:
                o.setdefault("MLUPS", {})[cp] = nc * sweeps_of(cp) * steps / (msm * 1e-3) / 1e6
                o.setdefault("speedup_vs_f64", {})[cp] = ms64 / msm
                near = near_cells(case["particles"][0], case["shape"])
                gbps = 2 * 19 * esize[m] * (nc - near) / (bulk * 1e-3) / 1e9
                o.setdefault("bulk_GBps", {})[cp] = gbps
                o.setdefault("frac", {})[cp] = gbps / peak
    out["f64"] = info
    if speed:
        shape = make_case(couplings[0])["shape"]
        out["workload"] = (f"settling sphere D=36, Ga=250 (nu=0.01), {shape[0]}x{shape[1]}x{shape[2]}, "
                           f"released at rest 64 cells below the top; {duration} lattice time units")
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1702_04910_gb300 import workloads as W
    from paper_1702_04910_gb300.binding import (PROFILE_CLASSES, Simulation, lbm_profile_enable,
                                                lbm_profile_read)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream().cuda_stream
    shape = workload(args.couplings[0], args.scale)["shape"]
    ncell = shape[0] * shape[1] * shape[2]

    def build(storage):
        sims = []
        for cp in args.couplings:
            case = workload(cp, args.scale)
            s = Simulation(case["shape"], stream=stream, storage=storage, **W.sim_kwargs(case))
            s.set_particles(case["particles"])
            s.init_equilibrium()
            sims.append(s)
        return sims

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(sims, steps, profile):
        for s in sims:
            lbm_profile_enable(s.h, profile)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(steps):
            for s in sims:
                s.step(1)
        ev1.record()
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        profs = [lbm_profile_read(s.h) if profile else None for s in sims]
        return ms, profs

    sweeps_per_step = sum(sweeps_of(c) for c in args.couplings)
    sims = build("f64")
    for _ in range(args.warmup):
        for s in sims:
            s.step(1)
    with ClockSampler(local) as clk:
        ms, profs = timed(sims, args.steps, True)
    clocks = clk.summary()
    value = job_mlups(world, ncell, sweeps_per_step, args.steps, ms * 1e-3)

    # dominant kernel: the bulk sweep (events recorded on the library's stream)
    bulk_ms = sum(p["bulk"][0] for p in profs)
    bulk_n = sum(p["bulk"][1] for p in profs)
    launches = sum(sum(v[1] for v in p.values()) for p in profs)
    share = {k: sum(p[k][0] for p in profs) for k in PROFILE_CLASSES}
    tot = sum(share.values())
    parts_now = [s.get_particles()[0] for s in sims]
    near = [near_cells(p, shape) for p in parts_now]
    bulk_cells = sum((ncell - nc) * sweeps_of(c) for nc, c in zip(near, args.couplings)) / sweeps_per_step
    bytes_per_cell = 2 * 19 * 8
    achieved = bytes_per_cell * bulk_cells / (bulk_ms / bulk_n * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()

    # end-to-end through the C ABI with host buffers: per step, the particle
    # state goes host -> device and forces + particle state come back
    e2e_sims = sims
    h2d = d2h = 0
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in e2e_sims:
            p = s.get_particles()
            s.set_particles(p)
            s.step(1)
            F, T = s.forces()
            h2d += 11 * 8 + 8
            d2h += 2 * (11 * 8 + 8) + F.nbytes + T.nbytes
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = job_mlups(world, ncell, sweeps_per_step, args.steps, e2e_s)

    # FP64 storage with the collision of cells away from particles in
    # float-float or 64-bit fixed-point arithmetic, FP32 and shifted 16-bit
    # storage: speed of the same timed step
    variants = {}
    for s in sims:
        s.close()
    sims = []
    what = {"f64ff": (8, "float-float (2 x FP32) collision away from particles, FP64 elsewhere"),
            "f64fx": (8, "64-bit fixed-point (2^-58) collision away from particles, FP64 elsewhere"),
            "f32": (4, "FP32 PDFs, FP32 collision"),
            "f16s": (2, "FP16 shifted populations f - w_q, FP32 collision"),
            "bf16s": (2, "BF16 shifted populations f - w_q, FP32 collision")}
    modes = [] if args.no_fp32 else ["f64fx", "f64ff", "f32", "f16s", "bf16s"]
    for mode in modes:
        esize, desc = what[mode]
        simsm = build(mode)
        for _ in range(args.warmup):
            for s in simsm:
                s.step(1)
        msm, profsm = timed(simsm, args.steps, True)
        vm = job_mlups(world, ncell, sweeps_per_step, args.steps, msm * 1e-3)
        bm = sum(p["bulk"][0] for p in profsm) / sum(p["bulk"][1] for p in profsm)
        achm = 2 * 19 * esize * bulk_cells / (bm * 1e-3) / 1e9
        for s in simsm:
            s.close()
        variants[mode] = {"value": vm, "unit": "MLUPS", "ms_per_step": msm / args.steps,
                          "speedup_vs_f64": vm / value, "bulk_GBps": achm, "frac": achm / peak,
                          "bulk_avg_launch_ms": bm, "algorithmic_bytes_per_cell": 2 * 19 * esize,
                          "arithmetic": desc}

    # settling-velocity and force error of each mode against the FP64 run of
    # the same case, as windowed means after release (the metric's "force /
    # velocity error vs FP64"), on this workload and on the D = 36, Ga = 250
    # case in 192 x 192 x 768
    if args.acc_time > 0 and modes:
        acc_modes = [m for m in modes if m != "f64ff"]
        acc = settling_errors(lambda cp: workload(cp, args.scale), args.couplings, acc_modes,
                              args.acc_time, stream)
        variants["settling_f64_reference"] = acc.pop("f64")
        for mode in acc_modes:
            variants[mode].update(acc[mode])
    if args.d36_time > 0 and not args.no_fp32:
        variants["settling_d36_ga250"] = settling_errors(
            lambda cp: W.settling_sphere(D=36.0, shape=(192, 192, 768), ga=250.0,
                                         drop_below_top=64.0, coupling=cp),
            ("PSM_M2B2", "MEM_CLI"), ["f64fx", "f16s", "bf16s"], args.d36_time, stream,
            speed=True, peak=peak)

    if not args.no_ensemble:
        variants.update(run_ensemble(args, stream, world, dist, barrier, peak))
    if args.learned != "none" and world == 1:
        variants[f"learned_{args.learned}"] = run_learned(args, stream)

    # dominant kernel's roofline against the metric's own bound, HBM bytes per
    # cell update; the kernel's actual limiter, the FP64 pipe, beside it with
    # the DFMA rate measured on this device
    from paper_1702_04910_gb300.binding import lbm_measure_fp64_rate
    props = torch.cuda.get_device_properties(local)
    sm_max_mhz = clocks.get("sm_max_mhz") or 2070.0
    fp64_nominal = FP64_LANE_OPS_PER_SM_CLK * props.multi_processor_count * sm_max_mhz * 1e6 / 1e12
    try:
        fp64_peak, fp64_src = lbm_measure_fp64_rate(stream) / 1e12, "measured (lbm_measure_fp64_rate)"
    except Exception as e:  # noqa: BLE001 - report the nominal figure instead
        fp64_peak, fp64_src = fp64_nominal, f"nominal ({e})"
    launch_s = bulk_ms / bulk_n * 1e-3
    fp64_achieved = K_BULK_F64_DP_INST_PER_CELL * bulk_cells / launch_s / 1e12
    traffic = (None if K_BULK_F64_DRAM_BYTES_PER_CELL is None
               else K_BULK_F64_DRAM_BYTES_PER_CELL * bulk_cells)
    roofline = {
        "bound": "hbm", "kernel": "k_bulk (fused pull stream + TRT collide), FP64",
        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "peak_source": peak_kind, "traffic": traffic,
        "per_unit": f"{bytes_per_cell} B per cell update (19 FP64 values read, 19 written)",
        "cells_per_launch": bulk_cells, "avg_launch_ms": bulk_ms / bulk_n,
        "limiter": "FP64 pipe (see alu): the kernel issues FP64 instructions at "
                   f"{fp64_achieved / fp64_peak:.2f} of the measured DFMA rate",
        "alu": {"achieved": fp64_achieved, "peak": fp64_peak, "unit": "T FP64 inst/s",
                "frac": fp64_achieved / fp64_peak, "peak_source": fp64_src,
                "peak_nominal": fp64_nominal,
                "peak_nominal_source": f"{FP64_LANE_OPS_PER_SM_CLK} FP64 lane-ops/SM/cycle x "
                                       f"{props.multi_processor_count} SMs x {sm_max_mhz:.0f} MHz",
                "per_unit": f"{K_BULK_F64_DP_INST_PER_CELL} FP64 instructions per cell update "
                            f"issued (ncu); {K_BULK_F64_DP_OPS_WRITTEN} written in the source"},
    }

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_steps, args.scale)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded workload, no dataset)",
            "config": {"workload": WORKLOAD if args.scale == 1.0 else f"{WORKLOAD} (scaled by {args.scale})",
                       "shape": list(shape), "couplings": list(args.couplings),
                       "lbm_sweeps_per_step": sweeps_per_step,
                       # the same rate counted per global step (one step of each coupling,
                       # MEM's two sweeps counted once): value x couplings / sweeps
                       "mlups_per_global_step": value * len(args.couplings) / sweeps_per_step,
                       "collision": "TRT (Lambda=3/16)",
                       "precision": "FP64 PDFs and collision; FP64 forces and rigid-body update",
                       "l2": "inputs larger than L2 (2.55 GB of PDFs per simulation)",
                       "replicas_per_rank": 1},
            "roofline": roofline,
            "kernel_time_share": {k: (v / tot if tot else 0.0) for k, v in share.items()},
            "kernel_time_share_note": "CUDA-event time per class; the near sweep runs on its own "
                                      "stream beside the bulk sweep, so its time includes the overlap",
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d // args.steps,
                    "d2h_bytes_per_step": d2h // args.steps,
                    "path": "C ABI per step: lbm_get_particles/lbm_set_particles (host), lbm_step, lbm_get_forces (host)"},
            "gpu_launches": launches,
            "clocks": clocks,
            "variants": variants,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def oracle_threads() -> int:
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env else (os.cpu_count() or 1)


def oracle_sample_step(sims):
    for o in sims:
        o.step(1)


def build_oracles(scale: float = 1.0):
    from oracle.oracle import Oracle
    from paper_1702_04910_gb300 import workloads as W
    sims = []
    for cp in COUPLINGS:
        case = workload(cp, scale)
        o = Oracle(case["shape"], **W.sim_kwargs(case))
        o.set_particles(case["particles"])
        o.init_equilibrium()
        sims.append(o)
    return sims


def cpu_baseline(steps: int, scale: float = 1.0):
    """The FP64 oracle (as it stands) on the same workload: `steps` global steps
    of the five variants on the full domain, host cores."""
    sims = build_oracles(scale)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_sample_step(sims)
    dt = time.perf_counter() - t0
    sweeps = sum(sweeps_of(c) for c in COUPLINGS)
    shape = sims[0].shape
    ncell = shape[0] * shape[1] * shape[2]
    for o in sims:
        o.close()
    return {"value": ncell * sweeps * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle_threads(),
            "kind": "oracle",
            "sample": f"{steps} global step(s) of the five variants on the full 128x128x512 domain "
                      f"({steps * sweeps} sweeps, {dt:.1f} s)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sims = build_oracles(args.scale)
    for _ in range(args.warmup):
        oracle_sample_step(sims)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(sims)
    dt = time.perf_counter() - t0
    sweeps = sum(sweeps_of(c) for c in COUPLINGS)
    shape = sims[0].shape
    ncell = shape[0] * shape[1] * shape[2]
    value = ncell * sweeps * args.steps / dt / 1e6
    world = int(os.environ.get("WORLD_SIZE", "1"))
    sample = (f"each step: one global step of the five variants on the full 128x128x512 domain "
              f"({sweeps} sweeps)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded workload, no dataset)",
            "config": {"workload": WORKLOAD if args.scale == 1.0 else f"{WORKLOAD} (scaled by {args.scale})",
                       "shape": list(shape), "couplings": list(COUPLINGS),
                       "lbm_sweeps_per_step": sweeps},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    for o in sims:
        o.close()
    print(json.dumps(line), flush=True)


def run_case(args):
    """Small profiling case: one simulation of --case-shape, --steps steps
    after --warmup (used for ncu captures of single kernels)."""
    import torch

    from paper_1702_04910_gb300 import workloads as W
    from paper_1702_04910_gb300.binding import Simulation
    shape = tuple(int(v) for v in args.case_shape.split("x"))
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    out = {}
    for cp in args.couplings:
        case = W.settling_sphere(shape=shape, drop_below_top=min(64.0, shape[2] / 2), coupling=cp)
        s = Simulation(case["shape"], stream=stream, storage=args.case_storage, **W.sim_kwargs(case))
        s.set_particles(case["particles"])
        s.init_equilibrium()
        s.step(args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(args.steps)
        s.synchronize()
        dt = time.perf_counter() - t0
        out[cp] = shape[0] * shape[1] * shape[2] * sweeps_of(cp) * args.steps / dt / 1e6
        s.close()
    print(json.dumps({"case": args.case_shape, "storage": args.case_storage, "MLUPS": out}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--couplings", default=None,
                    help="comma list; default PSM_M1B1,PSM_M2B2,MEM_BB,MEM_CLI,MEM_MR (the "
                         "settling step; the same five with --frame)")
    ap.add_argument("--acc-time", type=int, default=2400,
                    help="lattice time units after release of the FP64 / storage-mode accuracy "
                         "runs (errors are windowed means over the last third; 0 skips them)")
    ap.add_argument("--d36-time", type=int, default=2000,
                    help="lattice time units of the D = 36, Ga = 250 settling case (192x192x768) "
                         "run in FP64, F64_FX, FP16 and BF16 shifted storage (0 skips it)")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-cases", type=int, default=64)
    ap.add_argument("--ensemble-only", action="store_true",
                    help="time only the batched ensemble (one JSON object of variants)")
    ap.add_argument("--ensemble-storage", default="f64,f64fx")
    ap.add_argument("--learned", choices=("small", "full", "none"), default="small",
                    help="learned force correction study reported as a variant")
    ap.add_argument("--learned-only", action="store_true")
    ap.add_argument("--frame", type=float, default=None, metavar="D",
                    help="run the paper's benchmark frame (case A, Ga = 144) at diameter D for "
                         "MEM BB/CLI/MR and PSM M1B1/M2B2/M3B2 and print u_pV against the paper's "
                         "Tab. 1")
    ap.add_argument("--frame-ga", type=float, default=144.0,
                    help="Galileo number of the frame study (144: case A, compared with Tab. 1)")
    ap.add_argument("--frame-upv-ref", type=float, default=-1.285,
                    help="reference u_pV that sets the inflow Reynolds number |u_pV| Ga")
    ap.add_argument("--frame-subcycles", type=int, default=2,
                    help="LBM sweeps per step of every coupling in the frame, forces averaged "
                         "(Sec. 4.1: 2)")
    ap.add_argument("--frame-storage", default="f64fx",
                    choices=("f64", "f64fx", "f64ff", "f32", "f16s", "bf16s"))
    ap.add_argument("--lab-drag", action="store_true",
                    help="drag of a fixed sphere in an inflow against a sphere translating "
                         "through fluid at rest at the same relative speed (D = 24)")
    ap.add_argument("--lab-drag-windows", type=int, default=60)
    ap.add_argument("--remap-charge", action="store_true",
                    help="--lab-drag / --full-settling: MEM runs charge the momentum of covered "
                         "and uncovered cells to the particle (lbm_set_remap_charge)")
    ap.add_argument("--full-settling", action="store_true",
                    help="run the settling workload for --full-steps global steps per coupling "
                         "and report wall contact and stability")
    ap.add_argument("--full-steps", type=int, default=20000)
    ap.add_argument("--full-storage", default="f64fx",
                    choices=("f64", "f64fx", "f64ff", "f32", "f16s", "bf16s"))
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the settling workload by this factor in every length (tests)")
    ap.add_argument("--case-shape", default=None,
                    help="run a single small profiling case of this shape (e.g. 128x128x256)")
    ap.add_argument("--case-storage", default="f64",
                    choices=("f64", "f32", "f64ff", "f64fx", "f16s", "bf16s"))
    args = ap.parse_args()
    args.frame_couplings = FRAME_COUPLINGS
    if args.couplings is None:
        args.couplings = COUPLINGS
    else:
        args.couplings = tuple(c for c in args.couplings.split(",") if c)
        args.frame_couplings = args.couplings
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.case_shape:
        run_case(args)
    elif args.lab_drag and args.impl == "ours":
        run_lab_drag(args)
    elif args.full_settling and args.impl == "ours":
        run_full_settling(args)
    elif args.ensemble_only and args.impl == "ours":
        run_ensemble_only(args)
    elif args.frame is not None and args.impl == "ours":
        run_frame_study(args)
    elif args.learned_only and args.impl == "ours":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_learned(args, torch.cuda.current_stream().cuda_stream)), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
