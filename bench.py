#!/usr/bin/env python3
"""Benchmark of the PIC-DSMC particle pipeline on one GB300 (or N replicas).

Workload (the DSMC collision microbench): 1024 x 1024 Cartesian cells of
50 nm with periodic walls and no field, 1e8 super-particles -- Cu with a
lognormal(ln 1e23 m^-3, 1) density per cell, Cu+ 10 % of Cu, electrons equal
to Cu+ with a per-cell temperature uniform in [5, 50] eV, heavies at 2000 K --
all five electron-impact channels, FP32 state, dt = 1 fs.  One step = push +
deposit + cell sort + NTC collisions + spawn, over every particle.

Metric: particle-updates/s (particles advanced by push + sort + collide per
second).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain restatement of the method)
on a bounded sample of the same workload on this machine's host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s (sort+DSMC+push+deposit)"
UNIT = "particle-updates/s"
FALLBACK_HBM_GBS = 6800.0


def workload_desc(nz, nr, total):
    return (f"DSMC collision microbench: {nz}x{nr} Cartesian cells (50 nm, periodic, no field), "
            f"{total:.3g} super-particles (Cu lognormal(ln 1e23 m^-3, 1), Cu+ 10% of Cu, e = Cu+, "
            f"Te U[5,50] eV, heavies 2000 K), 5 channels incl. double ionization, FP32 state, dt = 1 fs")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nz", type=int, default=1024)
    p.add_argument("--nr", type=int, default=1024)
    p.add_argument("--total", type=float, default=1e8)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-rows", type=int, default=512, help="rows of cells in the CPU-baseline sample")
    p.add_argument("--cpu-steps", type=int, default=10)
    return p.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, x, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path):
        self.path = path
        self.p = None
        try:
            self.f = open(path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            v = d.get("hbm_gbs")
            if isinstance(v, dict):
                v = v.get("value")
            if v:
                return float(v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


# algorithmic bytes per live particle (FP32 SoA, 28 B per particle), per
# kernel, Cartesian field-free microbench
BYTES_PER_PARTICLE = {
    "push": 32.0,      # read key, pz, pr, vz, vr (20 B); write key, pz, pr (12 B)
    "scatter": 56.0,   # read 7 x 4 B, write 7 x 4 B
}


def cpu_baseline(args, cfg_full, seed):
    """The oracle (float mirror, as it stands, one thread) on a bounded sample:
    the first `cpu_rows` rows of cells of the same workload recipe."""
    import oracle
    import synthetic
    rows = args.cpu_rows
    total = args.total * rows / args.nz
    cfg, parts = synthetic.microbench(nz=rows, nr=args.nr, total=total, seed=seed)
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(synthetic.standin_cross_sections())
    o.load(parts)
    o.prime()
    n0 = o.count()
    t0 = time.perf_counter()
    o.step(args.cpu_steps)
    dt = time.perf_counter() - t0
    n1 = o.count()
    upd = args.cpu_steps * 0.5 * (n0 + n1)
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{rows}x{args.nr} cells of the same recipe ({n0} particles), {args.cpu_steps} steps, "
                      f"{dt:.1f} s, single-threaded C oracle (float mirror)"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    cb = cpu_baseline(args, None, seed=1)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.cpu_steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(args.nz, args.nr, args.total) + " (bounded CPU sample)",
                       "nz": args.cpu_rows, "nr": args.nr},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import paper_2109_00214_gb300 as pd
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pd.load_library()
    seed = 1 + rank
    cfg, parts = synthetic.microbench(nz=args.nz, nr=args.nr, total=args.total, seed=seed)
    xs = synthetic.standin_cross_sections()
    n_in = len(parts["species"])

    # ---- device-resident run (value) -------------------------------------
    sim = pd.Simulation(cfg, xs, device=dev)
    keys = ("species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")
    dtens = {k: torch.from_numpy(parts[k]).to(dev) for k in keys}
    sim.load_device(dtens)
    del dtens
    torch.cuda.synchronize()
    sim.step(args.warmup)
    sim.synchronize()
    pd.pd_profile_read(sim.h)              # discard warm-up launch records
    pd.pd_profile_enable(sim.h, 1)
    n0 = sim.scalars()["n_particles"]
    stream = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if ws == 1 else str(local)
    sampler = ClockSampler(gpu_index if gpu_index.isdigit() else local,
                           os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out"))
                                        else "", f"clocks_rank{rank}.csv"))
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = pd.pd_profile_read(sim.h)
    pd.pd_profile_enable(sim.h, 0)
    n1 = sim.scalars()["n_particles"]
    sim.synchronize()
    ms_max = max_over_ranks(ws, ms, dev)
    updates = args.steps * 0.5 * (n0 + n1)
    total_updates = sum_over_ranks(ws, updates, dev)
    value = total_updates / (ms_max * 1e-3)
    launches = int(sum(v[1] for v in prof.values()))

    # roofline of the dominant kernel (largest time share in the timed region)
    peak, peak_kind = peaks()
    dom = max(("push", "scatter"), key=lambda k: prof[k][0])
    per_launch_ms = prof[dom][0] / max(prof[dom][1], 1)
    bytes_per_launch = BYTES_PER_PARTICLE[dom] * 0.5 * (n0 + n1)
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    total_kernel_ms = sum(v[0] for v in prof.values())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
                "traffic": None, "algorithmic_bytes_per_launch": bytes_per_launch,
                "launch_ms": per_launch_ms,
                "share": prof[dom][0] / total_kernel_ms if total_kernel_ms > 0 else None,
                "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]}}
    counters = sim.counters()
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # ---- end-to-end through the public API with host buffers -------------
    e2e = None
    if not args.no_e2e:
        sim2 = pd.Simulation(cfg, xs, device=dev)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.load(parts)                    # host -> device inside the timed region
        sim2.step(args.steps)
        sc = sim2.scalars()                 # device -> host read of the result
        t1 = time.perf_counter()
        barrier(ws)
        wall = max_over_ranks(ws, t1 - t0, dev)
        upd2 = sum_over_ranks(ws, args.steps * 0.5 * (n_in + sc["n_particles"]), dev)
        h2d = 28 * n_in
        d2h = 1024 + 5 * 8
        e2e = {"value": upd2 / wall, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps}
        sim2.close()
        del sim2
        torch.cuda.empty_cache()

    cb = None
    if rank == 0 and not args.no_cpu and ws == 1:
        cb = cpu_baseline(args, cfg, seed=1)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_desc(args.nz, args.nr, args.total), "nz": args.nz, "nr": args.nr,
                           "particles_per_gpu": int(n0), "parallelism": f"replicas x{ws}" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (28 B x particles resident in HBM); no flush"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks,
                "events": {k: counters[k] for k in ("ev_el", "ev_exc", "ev_si", "ev_di", "ev_sw", "cand_total")}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
