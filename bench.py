#!/usr/bin/env python3
"""Benchmark of the coupled D3Q19 step on the 128 x 128 x 512 settling-sphere
workload (D = 24, density ratio 1.5, Galileo number 144, closed top and bottom).

One benchmark step is one global time step of each coupling variant that
stays stable for a freely settling sphere (PSM M1B1, M2B2: one LBM sweep each;
MEM BB, CLI: two LBM sweeps each, with refilling), each in its own simulation,
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
COUPLINGS = ("PSM_M1B1", "PSM_M2B2", "MEM_BB", "MEM_CLI")
SHAPE = (128, 128, 512)
WORKLOAD = ("settling sphere 128x128x512, D=24, rho_p/rho_f=1.5, Ga=144 (nu=0.01, tau=0.53), "
            "periodic x/y, no-slip z, released at rest 64 cells below the top; one global step "
            "of each of PSM M1B1/M2B2 (1 sweep) and MEM BB/CLI (2 sweeps, refilling)")
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


def near_tile_cells(particle, shape, tx, ty, halo=2.0):
    """Cells of the tiles the near-particle kernel takes (host restatement of
    the library's tiling: tx x ty x 1 tiles, sphere region R + halo)."""
    import numpy as np
    nx, ny, nz = shape
    R = 0.5 * particle["diameter"]
    count = 1
    for a, (n, T, periodic) in enumerate(((nx, tx, True), (ny, ty, True), (nz, 1, False))):
        X = particle["x"][a]
        lo = math.ceil(X - R - halo - 0.5)
        hi = math.floor(X + R + halo - 0.5)
        cells = np.arange(lo, hi + 1)
        cells = np.mod(cells, n) if periodic else cells[(cells >= 0) & (cells < n)]
        tiles = np.unique(cells // T)
        count *= sum(min(T, n - t * T) for t in tiles)
    return int(count)


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
    ncell = SHAPE[0] * SHAPE[1] * SHAPE[2]

    def build(storage):
        sims = []
        for cp in args.couplings:
            case = W.settling_sphere(coupling=cp)
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
        ms = ev0.elapsed_time(ev1)
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
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
    value = world * ncell * sweeps_per_step * args.steps / (ms * 1e-3) / 1e6

    # dominant kernel: the bulk sweep (events recorded on the library's stream)
    bulk_ms = sum(p["bulk"][0] for p in profs)
    bulk_n = sum(p["bulk"][1] for p in profs)
    launches = sum(sum(v[1] for v in p.values()) for p in profs)
    share = {k: sum(p[k][0] for p in profs) for k in PROFILE_CLASSES}
    tot = sum(share.values())
    tx = 128 if SHAPE[0] >= 128 else (64 if SHAPE[0] >= 64 else 32)
    ty = 256 // tx
    parts_now = [s.get_particles()[0] for s in sims]
    near = [near_tile_cells(p, SHAPE, tx, ty) for p in parts_now]
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
    e2e_s = time.perf_counter() - t0
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * ncell * sweeps_per_step * args.steps / e2e_s / 1e6

    # FP64 storage with the collision of cells away from particles in
    # float-float or 64-bit fixed-point arithmetic: speed and error against FP64
    variants = {}
    for s in sims:
        s.close()
    sims = []
    arith = {"f64ff": "float-float (2 x FP32) collision away from particles, FP64 elsewhere",
             "f64fx": "64-bit fixed-point (2^-58) collision away from particles, FP64 elsewhere"}
    for mode in ([] if args.no_fp32 else ["f64fx", "f64ff"]):
        simsm = build(mode)
        for _ in range(args.warmup):
            for s in simsm:
                s.step(1)
        msm, profsm = timed(simsm, args.steps, True)
        vm = world * ncell * sweeps_per_step * args.steps / (msm * 1e-3) / 1e6
        bm = sum(p["bulk"][0] for p in profsm) / sum(p["bulk"][1] for p in profsm)
        achm = bytes_per_cell * bulk_cells / (bm * 1e-3) / 1e9
        for s in simsm:
            s.close()
        s64, sm = build("f64"), build(mode)
        for a, b in zip(s64, sm):
            a.step(args.acc_steps)
            b.step(args.acc_steps)
        ferr, verr, perr = {}, {}, {}
        for c, a, b in zip(args.couplings, s64, sm):
            Fa, _ = a.forces()
            Fb, _ = b.forces()
            pa, pb = a.get_particles()[0], b.get_particles()[0]
            ferr[c] = float(np.linalg.norm(Fb - Fa) / max(np.linalg.norm(Fa), 1e-300))
            verr[c] = float(np.linalg.norm(pb["u"] - pa["u"]) / max(np.linalg.norm(pa["u"]), 1e-300))
            fa, fb = a.pdf(), b.pdf()
            perr[c] = float(np.max(np.abs(fb - fa)) / np.max(np.abs(fa)))
        variants[mode] = {"value": vm, "unit": "MLUPS", "ms_per_step": msm / args.steps,
                          "bulk_GBps": achm, "frac": achm / peak, "bulk_avg_launch_ms": bm,
                          "arithmetic": arith[mode], "pdf_max_rel_err_vs_f64": perr,
                          "force_rel_err_vs_f64": ferr, "particle_velocity_rel_err_vs_f64": verr,
                          "after_steps": args.acc_steps}
        for s in s64 + sm:
            s.close()

    # FP32 storage variant and its force / velocity error against FP64
    if not args.no_fp32:
        sims64 = build("f64")
        sims32 = build("f32")
        for _ in range(args.warmup):
            for s in sims32:
                s.step(1)
        ms32, profs32 = timed(sims32, args.steps, True)
        v32 = world * ncell * sweeps_per_step * args.steps / (ms32 * 1e-3) / 1e6
        b32 = sum(p["bulk"][0] for p in profs32) / sum(p["bulk"][1] for p in profs32)
        ach32 = 2 * 19 * 4 * bulk_cells / (b32 * 1e-3) / 1e9
        # accuracy: fresh pair, same start, args.acc_steps steps
        for s in sims32:
            s.close()
        sims32 = build("f32")
        nacc = args.acc_steps
        for s64, s32 in zip(sims64, sims32):
            s64.step(nacc)
            s32.step(nacc)
        ferr, verr = {}, {}
        for c, s64, s32 in zip(args.couplings, sims64, sims32):
            F64, _ = s64.forces()
            F32, _ = s32.forces()
            p64, p32 = s64.get_particles()[0], s32.get_particles()[0]
            ferr[c] = float(np.linalg.norm(F32 - F64) / max(np.linalg.norm(F64), 1e-300))
            verr[c] = float(np.linalg.norm(p32["u"] - p64["u"]) / max(np.linalg.norm(p64["u"]), 1e-300))
        variants["f32"] = {"value": v32, "unit": "MLUPS", "ms_per_step": ms32 / args.steps,
                           "bulk_GBps": ach32, "frac": ach32 / peak,
                           "force_rel_err_vs_f64": ferr, "particle_velocity_rel_err_vs_f64": verr,
                           "after_steps": nacc}
        for s in sims64 + sims32:
            s.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_steps)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded workload, no dataset)",
            "config": {"workload": WORKLOAD, "shape": list(SHAPE), "couplings": list(args.couplings),
                       "lbm_sweeps_per_step": sweeps_per_step, "collision": "TRT (Lambda=3/16)",
                       "precision": "FP64 PDFs and collision; FP64 forces and rigid-body update",
                       "l2": "inputs larger than L2 (2.55 GB of PDFs per simulation)",
                       "replicas_per_rank": 1},
            "roofline": {"bound": "hbm", "kernel": "k_bulk (fused pull stream + TRT collide)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "algorithmic_bytes_per_cell": bytes_per_cell,
                         "cells_per_launch": bulk_cells,
                         "avg_launch_ms": bulk_ms / bulk_n, "traffic": None},
            "kernel_time_share": {k: (v / tot if tot else 0.0) for k, v in share.items()},
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


def build_oracles():
    from oracle.oracle import Oracle
    from paper_1702_04910_gb300 import workloads as W
    sims = []
    for cp in COUPLINGS:
        case = W.settling_sphere(coupling=cp)
        o = Oracle(case["shape"], **W.sim_kwargs(case))
        o.set_particles(case["particles"])
        o.init_equilibrium()
        sims.append(o)
    return sims


def cpu_baseline(steps: int):
    """The FP64 oracle (as it stands) on the same workload: `steps` global steps
    of the five variants on the full 128x128x512 domain, host cores."""
    sims = build_oracles()
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_sample_step(sims)
    dt = time.perf_counter() - t0
    sweeps = sum(sweeps_of(c) for c in COUPLINGS)
    ncell = SHAPE[0] * SHAPE[1] * SHAPE[2]
    for o in sims:
        o.close()
    return {"value": ncell * sweeps * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle_threads(),
            "kind": "oracle",
            "sample": f"{steps} global step(s) of the four variants on the full 128x128x512 domain "
                      f"({steps * sweeps} sweeps, {dt:.1f} s)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sims = build_oracles()
    for _ in range(args.warmup):
        oracle_sample_step(sims)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(sims)
    dt = time.perf_counter() - t0
    sweeps = sum(sweeps_of(c) for c in COUPLINGS)
    ncell = SHAPE[0] * SHAPE[1] * SHAPE[2]
    value = ncell * sweeps * args.steps / dt / 1e6
    world = int(os.environ.get("WORLD_SIZE", "1"))
    sample = (f"each step: one global step of the four variants on the full 128x128x512 domain "
              f"({sweeps} sweeps)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded workload, no dataset)",
            "config": {"workload": WORKLOAD, "shape": list(SHAPE), "couplings": list(COUPLINGS),
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
    ap.add_argument("--couplings", default=",".join(COUPLINGS))
    ap.add_argument("--acc-steps", type=int, default=200)
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case-shape", default=None,
                    help="run a single small profiling case of this shape (e.g. 128x128x256)")
    ap.add_argument("--case-storage", default="f64", choices=("f64", "f32", "f64ff", "f64fx"))
    args = ap.parse_args()
    args.couplings = tuple(c for c in args.couplings.split(",") if c)
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.case_shape:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
