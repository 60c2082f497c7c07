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
  python bench.py --workload ensemble [--steps K] [--warmup W]
  python bench.py --workload warmstart

--workload warmstart trains the warm-start network on (rho, phi) pairs taken
every 2 steps from plume runs on 256^2 and 512^2 grids (runs split 90/10 into
training and held-out runs) and compares, on the held-out runs, the multigrid
cycles and step time to the residual tolerance from three starting points:
the charge-free potential (cold), the previous step's potential, and the
network's prediction.

--workload ensemble times the batched breakdown ensemble instead: 64 r-z runs
(8 seeds x gap voltages 2-10 kV, grids 64^2..256^2 cells, 1e5..2e6 particles
each, self-consistent Poisson field), advanced as one
ensemble under a CUDA graph with autotuned launch shapes, against the plain
method (the same 64 runs as separate simulations, one after another), both
with every Poisson solve at or below the same relative residual.

--workload stress is the microbench with the collision time step scaled
(--coll-scale, default 3200) so that a cell draws about one NTC candidate per
step: it exercises the collision, spawn and ordered candidate loop at full
size.  --workload production is the production-size breakdown: a 512 x 512
r-z plume of 2e7 particles (e, Cu, Cu2+ with SW/DI labels; 60 % ionized,
mean charge 2), self-consistent Poisson field to relres 1e-8 every step,
heavies on every 10th step.  Both report per-kernel times and algorithmic
GB/s.

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


def workload_desc(nz, nr, total, heavy_coll=0, coulomb=0, coll_scale=1.0):
    return (("DSMC collision microbench" if coll_scale == 1.0 else
             f"DSMC collision stress (microbench with the collision step x{coll_scale:g})")
            + f": {nz}x{nr} Cartesian cells (50 nm, periodic, no field), "
            f"{total:.3g} super-particles (Cu lognormal(ln 1e23 m^-3, 1), Cu+ 10% of Cu, e = Cu+, "
            f"Te U[5,50] eV, heavies 2000 K), 5 channels incl. double ionization"
            + (" + charge exchange and Cu-Cu elastic pairs" if heavy_coll else "")
            + (" + Coulomb e-e and e-ion pairs" if coulomb else "")
            + ", FP32 state, dt = 1 fs")


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
    p.add_argument("--workload", default="microbench",
                   choices=["microbench", "stress", "production", "ensemble", "warmstart"])
    p.add_argument("--coll-scale", type=float, default=None,
                   help="collision time step scale (stress: default 3200, about one candidate per cell)")
    p.add_argument("--prod-n", type=int, default=512, help="production: cells per side")
    p.add_argument("--prod-total", type=float, default=2e7, help="production: particles")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--eager", action="store_true",
                   help="time the eager steps only (the multigrid residual checked on the host), no CUDA graph")
    p.add_argument("--log-dir", default=".", help="where the clock samples of the timed region are written")
    p.add_argument("--heavy-coll", action="store_true",
                   help="microbench: add the heavy-particle pair classes (charge exchange, Cu-Cu elastic)")
    p.add_argument("--coulomb", action="store_true", help="microbench: add the Coulomb pair collisions")
    p.add_argument("--no-plain", action="store_true", help="ensemble: skip the one-simulation-per-run arm")
    p.add_argument("--ens-seeds", type=int, default=8, help="ensemble: seeds (runs = seeds x 8 voltages)")
    p.add_argument("--ens-warm", default="extrapolate", help="ensemble: Poisson starting point of every arm "
                   "(previous, extrapolate, cold)")
    p.add_argument("--ws-sizes", default="256,512", help="grid sizes of the warm-start runs")
    p.add_argument("--ws-runs", type=int, default=10, help="runs per grid size (the last one is held out)")
    p.add_argument("--ws-pairs", type=int, default=500, help="pairs per run, one every 2 steps")
    p.add_argument("--ws-particles", type=float, default=4e6, help="particles of a 512^2 run (scaled by area)")
    p.add_argument("--ws-iters", type=int, default=3000)
    p.add_argument("--ws-eval-steps", type=int, default=30)
    a = p.parse_args()
    if a.coll_scale is None:
        a.coll_scale = 3200.0 if a.workload == "stress" else 1.0
    if a.workload == "production" and "--steps" not in sys.argv:
        a.steps = 50
    if a.workload == "ensemble":
        if "--steps" not in sys.argv:
            a.steps = 40
        if "--warmup" not in sys.argv:
            a.warmup = 10
    return a


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


def shard(items, rank, ws):
    """The items rank `rank` of `ws` replicas takes (every ws-th, from its rank):
    the ranks' shares partition the items."""
    return items[rank::ws]


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


# DRAM bytes per live particle of the push from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of a launch of the 512 x 512
# microbench, 2.49e7 particles, the recipe of the 1024 x 1024 one), scaled to
# a launch by its particle count.  The figure holds only for the kernel source
# it was taken on: TRAFFIC_SOURCE_SHA is the push_source_digest() of the
# source at the capture, and `traffic` is null for any other source.
TRAFFIC_PER_PARTICLE = {"push": 796.619e6 / 24898326}
TRAFFIC_SOURCE_SHA = "4ea56a37e679cd6915a1f10f3105171b5066fd3f77c9b4c9d07c6f56dc5efaa0"
TRAFFIC_SOURCE = "ncu dram bytes per particle of a 2.49e7-particle launch, scaled"
PUSH_SECTION_END = "// sort: holes, insertions, re-layout"


def push_source_digest(read=None):
    """SHA-256 over the source the push kernel compiles from: csrc/pd_stream.cu
    up to its sort section (the push kernel and its helpers), its launcher
    launch_push, and the two headers its device code uses.  Edits elsewhere in
    the file (the sort kernels) and in the launchers' declarations leave it
    unchanged.  `read(relpath) -> str` supplies the files (default: the
    working tree)."""
    import hashlib
    csrc = "paper_2109_00214_gb300/csrc/"
    if read is None:
        def read(rel):
            with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
                return f.read()
    stream = read(csrc + "pd_stream.cu")
    cut = stream.find(PUSH_SECTION_END)
    start = stream.find("void launch_push(")
    end = stream.find("\n}\n", start)
    if cut < 0 or start < 0 or end < 0:
        return None
    h = hashlib.sha256()
    h.update(stream[:cut].encode())
    h.update(stream[start:end + 3].encode())
    for name in ("pd_internal.cuh", "pd_warp.cuh"):
        h.update(read(csrc + name).encode())
    return h.hexdigest()


def traffic_per_particle(kernel):
    try:
        sha = push_source_digest()
    except OSError:
        return None
    return TRAFFIC_PER_PARTICLE.get(kernel) if sha == TRAFFIC_SOURCE_SHA else None


def host_cpu():
    """Host cores the oracle uses and their model (lscpu's, else /proc/cpuinfo's)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return os.cpu_count() or 1, model


def cpu_baseline(args, cfg_full, seed, rows=None, steps=None, warmup=0):
    """The oracle (float mirror, as it stands, its OpenMP build on all host
    cores) on a bounded sample: the first `rows` rows of cells of the same
    workload recipe, `warmup` untimed steps, then `steps` timed ones."""
    import oracle
    import synthetic
    rows = args.cpu_rows if rows is None else rows
    steps = args.cpu_steps if steps is None else steps
    total = args.total * rows / args.nz
    cfg, parts = synthetic.microbench(nz=rows, nr=args.nr, total=total, seed=seed, coll_scale=args.coll_scale)
    if args.coll_scale != 1.0:
        cfg["capacity"] = int(2.0 * total) + 8 * rows * args.nr
    cfg["heavy_coll"] = int(args.heavy_coll)
    cfg["coulomb"] = int(args.coulomb)
    o = oracle.Oracle(cfg, fp64=False, omp=True)
    o.set_cross_sections(synthetic.standin_cross_sections())
    o.load(parts)
    o.prime()
    if warmup:
        o.step(warmup)
    n0 = o.count()
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    n1 = o.count()
    upd = steps * 0.5 * (n0 + n1)
    cores, model = host_cpu()
    return {"value": upd / dt, "unit": UNIT, "cores": cores, "cpu_model": model, "kind": "oracle",
            "ms_per_step": 1e3 * dt / steps,
            "sample": f"{rows}x{args.nr} cells of the same recipe ({n0} particles), {warmup} untimed and "
                      f"{steps} timed steps, {dt:.1f} s, C oracle (float mirror), OpenMP build on {cores} "
                      f"host cores"}


def cpu_baseline_production(args, seed, n=128, steps=None, warmup=1):
    """The oracle on a bounded sample of the production breakdown: the same
    plume recipe on an n x n grid with the particle total scaled by area
    (the oracle's conjugate-gradient solve of every step included)."""
    import oracle
    import synthetic
    steps = args.cpu_steps if steps is None else steps
    total = args.prod_total * (n / args.prod_n) ** 2
    cfg, parts = synthetic.rz_plume(n=n, total=total, seed=seed)
    cfg.update(field_on=1, inject_on=0, poisson_tol=1e-8)
    o = oracle.Oracle(cfg, fp64=False, omp=True)
    o.set_cross_sections(synthetic.standin_cross_sections())
    o.load(parts)
    o.prime()
    if warmup:
        o.step(warmup)

    def counts():
        return np.bincount(o.particles()["species"], minlength=7).astype(np.float64)

    c0 = counts()
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    c1 = counts()
    upd = step_updates(c0, c1, steps, cfg["heavy_subcycle"])
    cores, model = host_cpu()
    return {"value": upd / dt, "unit": UNIT, "cores": cores, "cpu_model": model, "kind": "oracle",
            "ms_per_step": 1e3 * dt / steps,
            "sample": f"the production plume recipe on {n}x{n} cells ({int(c0.sum())} particles), {warmup} untimed "
                      f"and {steps} timed steps, {dt:.1f} s, C oracle (float mirror, CG field solve), OpenMP build "
                      f"on {cores} host cores"}


def cpu_baseline_for(args, seed, steps=None, warmup=0, rows=None):
    if args.workload == "production":
        return cpu_baseline_production(args, seed, steps=steps, warmup=max(warmup, 1))
    return cpu_baseline(args, None, seed=seed, rows=rows, steps=steps, warmup=warmup)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    # the K timed steps (after W untimed ones) run on a sample of rows sized
    # for about ten 512-row steps of oracle time in all
    rows = max(8, min(args.cpu_rows, (args.cpu_rows * args.cpu_steps // max(args.steps, 1)) // 8 * 8))
    cb = cpu_baseline_for(args, seed=1, rows=rows, steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": single_workload_desc(args) + " (bounded CPU sample)",
                       "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


ENS_METRIC = "wall time per ensemble step at equal Poisson residual (64 breakdown runs)"


def ensemble_updates(c0, c1, steps, heavy_subcycle):
    """particle updates of `steps` steps: electrons every step, heavies on
    their sub-cycle steps (mean of the start and end populations)"""
    ne = 0.5 * (c0[0] + c1[0])
    nh = 0.5 * (sum(c0[1:]) + sum(c1[1:]))
    return steps * ne + (steps / heavy_subcycle) * nh


def run_ensemble(args, ws, rank, local):
    """Batched ensemble (one launch per kernel for all runs, CUDA graph,
    autotuned shapes) against the plain method (one simulation per run, run
    after run), at equal Poisson residual."""
    import torch
    import paper_2109_00214_gb300 as pd
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pd.load_library()
    all_runs = synthetic.ensemble_breakdown(seeds=range(1, args.ens_seeds + 1))
    runs = shard(all_runs, rank, ws)            # replicas: runs split across ranks, no collective
    xs = synthetic.standin_cross_sections()
    cfgs = [c for c, _ in runs]
    R = len(runs)
    tol = max(c["poisson_tol"] for c in cfgs)
    G = 2 * cfgs[0]["heavy_subcycle"] if cfgs[0]["heavy_subcycle"] % 2 else cfgs[0]["heavy_subcycle"]
    W = -(-args.warmup // G) * G
    K = -(-args.steps // G) * G
    hs = cfgs[0]["heavy_subcycle"]
    keys = ("species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")

    def counts(get):
        c = np.zeros(7)
        for r in range(R):
            c += np.array(get(r)["count"], dtype=np.float64)
        return c

    def timed(stream, fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        barrier(ws)
        return e0.elapsed_time(e1), (t1 - t0) * 1e3

    # ---- plain method: one simulation per run, run after run --------------
    plain_ms = plain_wall = plain_upd = None
    plain_relres = plain_eager = plain_cycles = None
    sims = [] if not args.no_plain else None
    if sims is not None:
        for cfg, parts in runs:
            sm = pd.Simulation(cfg, xs, device=dev)
            sm.set_warm_start(args.ens_warm)
            sm.load_device({k: torch.from_numpy(parts[k]).to(dev) for k in keys})
            sims.append(sm)
        for sm in sims:
            sm.step(W)
        torch.cuda.synchronize()
        # eager: host-checked multigrid, one launch sequence per run and step
        c0 = counts(lambda r: sims[r].scalars())
        eager_ms, eager_wall = timed(sims[0].stream, lambda: [sm.step(K) for sm in sims])
        plain_sc = [sm.scalars() for sm in sims]
        c1 = counts(lambda r: plain_sc[r])
        eager_upd = ensemble_updates(c0, c1, K, hs)
        eager_relres = max(sc["poisson_relres_max"] for sc in plain_sc)
        plain_eager = {"ms_per_step": max_over_ranks(ws, eager_ms, dev) / K, "wall_ms_per_step": eager_wall / K,
                       "poisson_relres_max": eager_relres,
                       "particle_updates_per_s": sum_over_ranks(ws, eager_upd, dev) /
                       (max_over_ranks(ws, eager_ms, dev) * 1e-3),
                       "method": "one simulation per run, stepped run after run, host-checked multigrid"}
        # each run under its own CUDA graph of G steps, a fixed cycle count
        # raised until every solve of the timed steps reaches the tolerance
        plain_cycles = int(max(sc["poisson_cycles"] for sc in plain_sc)) + 1
        for attempt in range(4):
            for sm in sims:
                sm.set_graph_mode(1, plain_cycles)
                sm.step(G)                       # capture + one replay, untimed
            torch.cuda.synchronize()
            c0 = counts(lambda r: sims[r].scalars())
            plain_ms, plain_wall = timed(sims[0].stream, lambda: [sm.step(K) for sm in sims])
            plain_sc = [sm.scalars() for sm in sims]
            plain_relres = max(sc["poisson_relres_max"] for sc in plain_sc)
            if plain_relres <= tol:
                break
            plain_cycles += 2
        c1 = counts(lambda r: plain_sc[r])
        plain_upd = ensemble_updates(c0, c1, K, hs)
        for sm in sims:
            sm.close()
        del sims
        torch.cuda.empty_cache()

    # ---- batched ensemble ---------------------------------------------------
    ens = pd.Ensemble(cfgs, xs, device=dev)
    ens.set_warm_start(args.ens_warm)
    for r, (_, parts) in enumerate(runs):
        ens.load_run_device(r, {k: torch.from_numpy(parts[k]).to(dev) for k in keys})
    tuning = None
    if not args.no_autotune:
        tuning = ens.autotune(4)
    # eager warm-up with host-checked solves; per-kernel times of the last G steps
    done = int(ens.run_scalars(0)["step"])      # steps the autotuner took
    ens.step(W + (G - (done + W) % G) % G)      # end on a multiple of the graph period
    ens.synchronize()
    pd.pd_profile_read(ens.h)
    pd.pd_profile_enable(ens.h, 1)
    ens.step(G)
    prof = pd.pd_profile_read(ens.h)
    pd.pd_profile_enable(ens.h, 0)
    cyc = max(ens.run_scalars(r)["poisson_cycles"] for r in range(R))
    # graph mode: a fixed cycle count; raised until every solve of the timed
    # steps reaches the tolerance
    cycles = int(cyc) + 1
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if ws == 1 else str(local)
    out_dir = args.log_dir
    for attempt in range(4):
        ens.set_graph_mode(1, cycles)
        ens.step(G)                              # capture + one replay, untimed
        ens.synchronize()
        pd.pd_profile_read(ens.h)
        c0 = counts(ens.run_scalars)
        sampler = ClockSampler(gpu_index if gpu_index.isdigit() else local,
                               os.path.join(out_dir, f"clocks_ensemble_rank{rank}.csv"))
        ens_ms, ens_wall = timed(ens.stream, lambda: ens.step(K))
        clocks = sampler.stop()
        launches = int(sum(n for _, n in pd.pd_profile_read(ens.h).values()))
        sc = [ens.run_scalars(r) for r in range(R)]
        relres = max(x["poisson_relres_max"] for x in sc)
        if relres <= tol:
            break
        cycles += 2
    c1 = counts(lambda r: sc[r])
    ens_upd = ensemble_updates(c0, c1, K, hs)
    nparts = int(sum(c1))
    ens.close()
    del ens
    torch.cuda.empty_cache()

    # ---- end to end: host loads, K graph steps, per-run scalars back ------
    e2e = None
    if not args.no_e2e:
        ens2 = pd.Ensemble(cfgs, xs, device=dev)
        ens2.set_warm_start(args.ens_warm)
        if tuning:
            ens2.set_tuning(**tuning)
        ens2.set_graph_mode(1, cycles)

        pinned = [{k: torch.from_numpy(np.ascontiguousarray(p[k])).pin_memory() for k in keys} for _, p in runs]

        def e2e_run():
            for r, pin in enumerate(pinned):
                pd.pd_load_particles_run_ptrs(ens2.h, r, pin["species"].numel(), [pin[k].data_ptr() for k in keys])
            ens2.step(K)
            return [ens2.run_scalars(r) for r in range(R)]
        _, wall = timed(ens2.stream, e2e_run)
        h2d = sum(29 * len(p["species"]) for _, p in runs)
        e2e = {"value": max_over_ranks(ws, wall, dev) / K, "unit": "ms/step",
               "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": R * 256 / K}
        ens2.close()
        del ens2
        torch.cuda.empty_cache()

    ens_ms_max = max_over_ranks(ws, ens_ms, dev)
    plain_ms_max = max_over_ranks(ws, plain_ms, dev) if plain_ms is not None else None
    upd_all = sum_over_ranks(ws, ens_upd, dev)
    if rank == 0:
        grids = {}
        for c in cfgs:
            grids[c["nz"]] = grids.get(c["nz"], 0) + 1
        line = {"metric": ENS_METRIC, "value": ens_ms_max / K, "unit": "ms/step", "n_gpus": ws, "steps": K,
                "warmup": W, "ms_per_step": ens_ms_max / K, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"batched breakdown ensemble: {len(all_runs)} r-z runs (8 seeds x "
                                       f"{len(synthetic.ENSEMBLE_VOLTS_KV)} gap voltages 2-10 kV), grids "
                                       f"{sorted(grids)} cells per side, 1e5..2e6 particles per run, "
                                       f"Poisson to relres <= {tol:g} from the {args.ens_warm} start, plume start without cathode "
                                       f"emission, dt = 1 fs",
                           "runs_per_gpu": R, "grid_histogram": grids, "particles_per_gpu": nparts,
                           "parallelism": f"runs split over {ws} replicas" if ws > 1 else "single",
                           "l2": "particle store larger than L2; no flush"},
                "batched": {"ms_per_step": ens_ms_max / K, "wall_ms_per_step": ens_wall / K,
                            "poisson_cycles_fixed": cycles, "poisson_relres_max": relres,
                            "particle_updates_per_s": upd_all / (ens_ms_max * 1e-3), "tuning": tuning,
                            "eager_kernels_ms_per_step": {k: v[0] / G for k, v in prof.items() if v[1]}},
                "plain": None if plain_ms is None else {
                    "ms_per_step": plain_ms_max / K, "wall_ms_per_step": plain_wall / K,
                    "poisson_relres_max": plain_relres, "poisson_cycles_fixed": plain_cycles,
                    "particle_updates_per_s": sum_over_ranks(ws, plain_upd, dev) / (plain_ms_max * 1e-3),
                    "method": "one simulation per run, stepped run after run, each under its own CUDA graph "
                              "of G steps with a fixed cycle count"},
                "plain_eager": plain_eager,
                "equal_residual": bool(relres <= tol and (plain_relres is None or plain_relres <= tol)),
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)


WS_METRIC = "Poisson multigrid cycles per step to relres 1e-8: cold vs previous-step vs extrapolated vs learned warm start"


def run_warmstart(args, ws, rank, local):
    import torch
    import paper_2109_00214_gb300 as pd
    from paper_2109_00214_gb300 import warmstart as W
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pd.load_library()
    xs = synthetic.standin_cross_sections()
    sizes = [int(v) for v in args.ws_sizes.split(",")]
    kinds = ("absolute", "delta", "extrap")
    mode_of = {"absolute": "learned", "delta": "learned_delta", "extrap": "learned_extrap"}
    t0 = time.perf_counter()
    sets = {k: [] for k in kinds}
    held = {k: {} for k in kinds}
    evals = {}
    for n in sizes:
        total = args.ws_particles * (n / 512.0) ** 2
        runs = []
        for k in range(args.ws_runs):
            cfg, parts = synthetic.rz_plume(n=n, total=total, seed=100 * n + k + 1)
            cfg.update(field_on=1, inject_on=0, run=k, V0=1e3 * (2 + (k % 8)), poisson_tol=1e-8)
            runs.append((cfg, parts))
        train_runs, test_runs = runs[:-1], runs[-1:]
        tr = W.collect_pairs([c for c, _ in train_runs], [p for _, p in train_runs], xs, args.ws_pairs,
                             kinds=kinds, device=dev)
        te = W.collect_pairs([c for c, _ in test_runs], [p for _, p in test_runs], xs, args.ws_pairs,
                             kinds=kinds, device=dev)
        for k in kinds:
            sets[k].append((tr[k][0].flatten(0, 1), tr[k][1].flatten(0, 1)))
            held[k][n] = (te[k][0].flatten(0, 1), te[k][1].flatten(0, 1))
        evals[n] = test_runs[0]
        del tr, te
    t_data = time.perf_counter() - t0
    # mini-batches of about 5.3e5 nodes (8 grids of 257^2, 2 of 513^2), at most 16 grids
    batch = [int(min(16, max(1, round(5.3e5 / (n + 1) ** 2)))) for n in sizes]
    max_nodes = max(b * (n + 1) ** 2 for b, n in zip(batch, sizes))
    rng = np.random.default_rng(1)
    p0 = []
    for ci, co in ((1, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 1)):
        p0.append(rng.standard_normal(9 * co * ci) * np.sqrt(2.0 / (9 * ci)))
        p0.append(np.zeros(co))
    p0 = np.concatenate(p0).astype(np.float32)
    nets, train_info = {}, {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for k in kinds:
        # the extrapolated form learns to cancel the residual its start leaves
        lk = "rz" if k == "extrap" else "mse"
        net = pd.Net(max_nodes, params=p0, device=dev)
        torch.cuda.synchronize()
        e0.record(net.stream)
        hist = W.train(net, sets[k], args.ws_iters, batch, lr=3e-3 if lk == "rz" else 1e-3, lr_final=5e-5,
                       log_every=max(1, args.ws_iters // 10), loss=lk)
        e1.record(net.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tl = {}
        for n, b in zip(sizes, batch):
            X, T = held[k][n]
            tl[str(n)] = {"test_loss": W.test_loss(net, X, T, batch=b, loss=lk),
                          "test_target_mean_square": float(torch.mean(T.double() ** 2).item())}
            if lk == "rz":
                # the same loss of the uncorrected start (y = 0): the mean square of w x
                w = torch.arange(n + 1, dtype=torch.float64, device=X.device)
                w[0], w[n] = 0.125, n / 2.0 - 0.125
                tl[str(n)]["loss_of_extrapolated_start"] = float(
                    torch.mean((X[:, 1:-1, :].double() * w) ** 2).item())
        train_info[k] = {"loss": lk, "loss_history": hist, "train_ms": ms,
                         "ms_per_iter": ms / max(args.ws_iters, 1), "held_out": tl}
        nets[mode_of[k]] = net
    modes = ("previous", "extrapolate", "cold", "learned", "learned_delta", "learned_extrap")
    results = {str(n): W.compare_starts(*evals[n], xs, nets, args.ws_eval_steps, modes=modes, device=dev)
               for n in sizes}
    # inference time on the largest grid
    n = max(sizes)
    net = nets["learned"]
    x1 = held["absolute"][n][0][:1].contiguous()
    for _ in range(3):
        net.forward(x1)
    e0.record(net.stream)
    for _ in range(20):
        net.forward(x1)
    e1.record(net.stream)
    torch.cuda.synchronize()
    infer_ms = e0.elapsed_time(e1) / 20
    flops = 2.0 * (n + 1) ** 2 * (9 * 32 * 2 + 4 * 9 * 32 * 32)
    big = results[str(n)]
    best = min(("learned", "learned_delta", "learned_extrap"), key=lambda m: big[m]["cycles_per_step"])
    if rank == 0:
        line = {"metric": WS_METRIC, "value": big[best]["cycles_per_step"], "unit": "cycles/step",
                "n_gpus": ws, "steps": args.ws_eval_steps, "warmup": 2,
                "ms_per_step": big[best]["ms_per_step"], "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 (network), f64 (solve)", "data": "synthetic",
                "config": {"workload": f"learned Poisson warm start: {len(sizes)} x {args.ws_runs} plume runs on "
                                       f"{sizes} grids, {args.ws_pairs} (rho, phi) pairs per run every 2 steps, "
                                       f"90/10 train/held-out split by run; 6 x conv3x3 (32 ch), bf16 weights, "
                                       f"fp32 accumulation; evaluated on the held-out {n}^2 run",
                           "pairs_per_kind": int(sum(x.shape[0] for x, _ in sets["absolute"]) +
                                                 sum(h[0].shape[0] for h in held["absolute"].values())),
                           "train_iters": args.ws_iters, "batch": batch, "value_mode": best},
                "results": results, "training": train_info, "data_s": t_data,
                "inference": {"grid": n, "ms": infer_ms, "tflops": flops / (infer_ms * 1e-3) / 1e12}}
        print(json.dumps(line), flush=True)
    for net in nets.values():
        net.close()


def single_workload_desc(args):
    if args.workload == "production":
        return (f"production breakdown: {args.prod_n}x{args.prod_n} r-z cells over the 6 um gap, "
                f"{args.prod_total:.3g} super-particles of a near-cathode Cu plume (e, Cu, Cu2+ SW/DI; 60 % "
                f"ionized, mean charge 2, Te 5 eV, heavies 2000 K), self-consistent Poisson field to relres "
                f"1e-8 every step (extrapolated start), heavies every 10th step, cathode emission off, FP32 "
                f"cell-relative state, int64 deposit, dt = 1 fs")
    return workload_desc(args.nz, args.nr, args.total, args.heavy_coll, args.coulomb, args.coll_scale)


def single_workload(args, seed):
    """(config, particles, description, warm-start mode) of the one-simulation workloads."""
    import synthetic
    if args.workload == "production":
        cfg, parts = synthetic.rz_plume(n=args.prod_n, total=args.prod_total, seed=seed)
        cfg.update(field_on=1, inject_on=0, poisson_tol=1e-8)
        return cfg, parts, single_workload_desc(args), "extrapolate"
    cfg, parts = synthetic.microbench(nz=args.nz, nr=args.nr, total=args.total, seed=seed,
                                      coll_scale=args.coll_scale)
    if args.coll_scale != 1.0:
        # about one candidate per cell reserves two spawn slots each per step,
        # and the ionizations add particles (a few per cent of the electrons
        # per step): room for both over the tuning, warm-up and timed steps
        cfg["capacity"] = int(2.0 * args.total) + 8 * args.nz * args.nr
    cfg["heavy_coll"] = int(args.heavy_coll)
    cfg["coulomb"] = int(args.coulomb)
    return cfg, parts, single_workload_desc(args), None


def step_updates(c0, c1, steps, heavy_subcycle):
    """Particle updates of `steps` steps from the species counts at their start
    and end: electrons every step, heavies on their sub-cycle steps."""
    return ensemble_updates(c0, c1, steps, heavy_subcycle)


def kernel_table(prof, steps, n_live, n_e, n_h, hs, slots, cand, ncell, nbins_h, rz_field, peak):
    """Per-kernel time per step and, where the kernel has a per-unit byte
    model, its algorithmic GB/s and fraction of the HBM peak.

    push: an electron's key, position and velocity are read (24 B, with
    v_theta, which the Cartesian push reads only for the record) with its id
    (4 B), and its record written to the mover buffer (28 B); a heavy
    particle on a heavy step is read and its new position written back
    (20 + 8 B Cartesian; 24 + 20 B r-z), on the other steps only its key is
    read (4 B); a slack slot reads its key (4 B).
    scatter (the sort after the push): every electron is read from the mover
    buffer and written to its bin (28 + 28 B); each heavy bin's in and out
    counts are read (8 B); heavy movers are few."""
    slack = max(slots - n_live, 0.0)
    if rz_field:
        heavy = n_h * (44.0 + 4.0 * (hs - 1)) / hs
        push_bytes = 56.0 * n_e + heavy + 4.0 * slack
    else:
        push_bytes = 56.0 * n_e + 28.0 * n_h + 4.0 * slack
    model = {
        "push": push_bytes,
        "scatter": 56.0 * n_e + 8.0 * nbins_h,
        "ncand": 24.0 * ncell,
        "collide": 100.0 * cand,
    }
    out = {}
    for k, (ms, n) in prof.items():
        if not n:
            continue
        row = {"ms_per_step": ms / steps, "launches_per_step": n / steps}
        if k in model and ms > 0:
            gbs = model[k] / (ms / steps * 1e-3) / 1e9
            row.update({"algorithmic_bytes_per_step": model[k], "GBs": gbs, "frac_of_peak": gbs / peak})
        out[k] = row
    return out


def run_single(args, ws, rank, local):
    """One simulation on one GPU (replicas: one per rank): the microbench, its
    stress variant or the production breakdown."""
    import torch
    import paper_2109_00214_gb300 as pd
    import synthetic

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pd.load_library()
    seed = 1 + rank
    cfg, parts, desc, warm = single_workload(args, seed)
    xs = synthetic.standin_cross_sections()
    n_in = len(parts["species"])
    hs = cfg["heavy_subcycle"]
    rz_field = cfg["geometry"] == "rz" and cfg["field_on"] == 1
    steps = args.steps
    if hs > 1:                 # whole heavy cycles
        steps = -(-steps // hs) * hs

    # ---- device-resident run (value) -------------------------------------
    sim = pd.Simulation(cfg, xs, device=dev)
    if warm:
        sim.set_warm_start(warm)
    keys = ("species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")
    dtens = {k: torch.from_numpy(parts[k]).to(dev) for k in keys}
    sim.load_device(dtens)
    del dtens
    torch.cuda.synchronize()
    tuning = None if args.no_autotune else sim.autotune(4)   # its trial steps are untimed warm-up
    done = int(sim.scalars()["step"])
    warm_steps = args.warmup + ((hs - (done + args.warmup) % hs) % hs if hs > 1 else 0)
    sim.step(warm_steps)
    sim.synchronize()
    pd.pd_profile_read(sim.h)              # discard warm-up launch records
    pd.pd_profile_enable(sim.h, 1)
    counters0 = sim.counters()
    sc0 = sim.scalars()
    ss0 = sim.sort_stats()
    n0 = sc0["n_particles"]
    stream = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if ws == 1 else str(local)
    sampler = ClockSampler(gpu_index if gpu_index.isdigit() else local,
                           os.path.join(args.log_dir, f"clocks_rank{rank}.csv"))
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    prof = pd.pd_profile_read(sim.h)
    pd.pd_profile_enable(sim.h, 0)
    sc1 = sim.scalars()
    n1 = sc1["n_particles"]
    sim.synchronize()
    ms_max = max_over_ranks(ws, ms, dev)
    c0 = np.array(sc0["count"], dtype=np.float64)
    c1 = np.array(sc1["count"], dtype=np.float64)
    updates = step_updates(c0, c1, steps, hs)
    total_updates = sum_over_ranks(ws, updates, dev)
    value = total_updates / (ms_max * 1e-3)
    launches = int(sum(v[1] for v in prof.values()))
    counters1 = sim.counters()
    counters = {k: counters1[k] - counters0[k] for k in counters1}   # events of the timed steps
    ss1 = sim.sort_stats()
    sort = {"relayouts_in_timed_steps": ss1["relayouts"] - ss0["relayouts"],
            "bin_slots_per_live_particle": ss1["bin_slots"] / max(ss1["live"], 1)}

    # roofline of the dominant kernel (largest time share in the timed region)
    peak, peak_kind = peaks()
    n_live = 0.5 * (n0 + n1)
    ne = 0.5 * (c0[0] + c1[0])
    nh = n_live - ne
    ncell = cfg["nz"] * cfg["nr"]
    nbins_h = ncell * (6 if cfg.get("charge_max", 2) >= 3 else 4)
    slots = float(ss1["bin_slots"])
    table = kernel_table(prof, steps, n_live, ne, nh, hs, slots, counters["cand_total"] / steps, ncell, nbins_h,
                         rz_field, peak)
    cands = [k for k in ("push", "scatter") if k in table and "GBs" in table[k]]
    dom = max(cands, key=lambda k: table[k]["ms_per_step"])
    per_launch_ms = prof[dom][0] / max(prof[dom][1], 1)
    bytes_per_launch = table[dom]["algorithmic_bytes_per_step"] / table[dom]["launches_per_step"]
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    total_kernel_ms = sum(v[0] for v in prof.values())
    tpp = None if (rz_field or args.coll_scale != 1.0) else traffic_per_particle(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
                "traffic": tpp * n_live if tpp else None,
                "traffic_source": TRAFFIC_SOURCE if tpp else None,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "launch_ms": per_launch_ms,
                "share": prof[dom][0] / total_kernel_ms if total_kernel_ms > 0 else None,
                "kernels_ms_per_step": {k: v["ms_per_step"] for k, v in table.items()}}
    poisson = None
    if rz_field:
        poisson = {"cycles_last": sc1["poisson_cycles"], "relres_max": sc1["poisson_relres_max"],
                   "tol": cfg["poisson_tol"], "warm_start": warm}

    # ---- the same steps as one CUDA graph per heavy cycle ------------------
    # A graph replays the step's launches without the host; with the field
    # on, the eager path checks the multigrid residual on the host after
    # every V-cycle, and a graph runs a fixed cycle count instead, raised
    # until every solve of the timed steps reaches the tolerance.  The faster
    # of the two timings is the headline; the per-kernel table above comes
    # from the eager pass.
    graph = None
    cycles = None
    if not args.eager:
        G = hs if hs % 2 == 0 else 2 * hs
        Kg = -(-steps // G) * G
        cycles = int(sc1["poisson_cycles"]) + 1
        for attempt in range(4):
            sim.set_graph_mode(1, cycles)
            done = int(sim.scalars()["step"])
            sim.step(G + (G - done % G) % G)           # capture + one replay, untimed
            sim.synchronize()
            pd.pd_profile_read(sim.h)
            g0 = np.array(sim.scalars()["count"], dtype=np.float64)
            sampler = ClockSampler(gpu_index if gpu_index.isdigit() else local,
                                   os.path.join(args.log_dir, f"clocks_graph_rank{rank}.csv"))
            barrier(ws)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(Kg)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier(ws)
            gclocks = sampler.stop()
            gms = e0.elapsed_time(e1)
            glaunch = int(sum(n for _, n in pd.pd_profile_read(sim.h).values()))
            gsc = sim.scalars()
            if gsc["poisson_relres_max"] <= cfg["poisson_tol"]:
                break
            cycles += 2
        gms_max = max_over_ranks(ws, gms, dev)
        g1 = np.array(gsc["count"], dtype=np.float64)
        gupd = sum_over_ranks(ws, step_updates(g0, g1, Kg, hs), dev)
        graph = {"value": gupd / (gms_max * 1e-3), "ms_per_step": gms_max / Kg, "steps": Kg,
                 "poisson_cycles_fixed": cycles if rz_field else None,
                 "poisson_relres_max": gsc["poisson_relres_max"],
                 "gpu_launches": glaunch, "clocks": gclocks,
                 "valid": bool(gsc["poisson_relres_max"] <= cfg["poisson_tol"])}
        graph["headline"] = graph["valid"] and graph["value"] > value
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # ---- end-to-end through the public API with host buffers -------------
    # the particle load is the run's input: it is copied host -> device once
    # per timed run of `steps` steps, and the scalars are read back at its end
    e2e = None
    if not args.no_e2e:
        sim2 = pd.Simulation(cfg, xs, device=dev)
        if warm:
            sim2.set_warm_start(warm)
        if tuning:
            sim2.set_tuning(**tuning)
        if graph is not None and graph["headline"]:
            sim2.set_graph_mode(1, cycles)
        # the inputs in pinned host memory (prepared outside the timed region)
        pinned = {k: torch.from_numpy(np.ascontiguousarray(parts[k])).pin_memory() for k in keys}
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pd.pd_load_particles_ptrs(sim2.h, n_in, [pinned[k].data_ptr() for k in keys])   # host -> device
        sim2.step(steps)
        sc = sim2.scalars()                 # device -> host read of the result
        t1 = time.perf_counter()
        barrier(ws)
        wall = max_over_ranks(ws, t1 - t0, dev)
        ce = np.zeros(7)
        for sp in range(7):
            ce[sp] = float(np.count_nonzero(parts["species"] == sp))
        upd2 = sum_over_ranks(ws, step_updates(ce, np.array(sc["count"], dtype=np.float64), steps, hs), dev)
        h2d = 29 * n_in                     # species 1 B, cell indices 2 x 4 B, offsets and velocities 5 x 4 B
        d2h = 1024 + 5 * 8
        e2e = {"value": upd2 / wall, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
               "d2h_bytes_per_step": d2h / steps,
               "copies": "particle load host -> device once per timed run of `steps` steps (pinned), "
                         "scalars device -> host at its end"}
        sim2.close()
        del sim2
        torch.cuda.empty_cache()

    cb = None
    if rank == 0 and not args.no_cpu and ws == 1:
        cb = cpu_baseline_for(args, seed=1)

    eager = None
    if graph is not None and graph["headline"]:
        # the headline is the graph run; the eager one explains it kernel by kernel
        eager = {"value": value, "ms_per_step": ms_max / steps, "steps": steps, "gpu_launches": launches,
                 "clocks": clocks, "poisson": poisson}
        value, ms_max, steps = graph["value"], graph["ms_per_step"] * graph["steps"], graph["steps"]
        launches, clocks = graph["gpu_launches"], graph["clocks"]
        if poisson is not None:
            poisson = dict(poisson, cycles_fixed=graph["poisson_cycles_fixed"],
                           relres_max=graph["poisson_relres_max"], mode="CUDA graph, fixed cycle count")
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
                "warmup": warm_steps, "ms_per_step": ms_max / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": desc, "nz": cfg["nz"], "nr": cfg["nr"],
                           "particles_per_gpu": int(n0), "parallelism": f"replicas x{ws}" if ws > 1 else "single",
                           "tuning": tuning,
                           "l2": "inputs larger than L2 (28 B x particles resident in HBM); no flush"},
                "roofline": roofline, "kernels": table, "sort": sort, "poisson": poisson, "cpu_baseline": cb,
                "timing": ("timed steps as CUDA graphs (one per heavy cycle); per-kernel table and roofline "
                           "from an eager pass of as many steps just before" if eager else
                           "eager launches; per-kernel CUDA events over the timed steps"),
                "eager": eager,
                "graph": None if graph is None or graph["headline"] else {
                    k: graph[k] for k in ("value", "ms_per_step", "steps", "valid")},
                "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "events": {k: counters[k] for k in ("ev_el", "ev_exc", "ev_si", "ev_di", "ev_sw", "ev_cx", "ev_nn",
                                                    "coul_ee", "coul_ei", "cand_total")}}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload in ("ensemble", "warmstart"):
        (run_ensemble if args.workload == "ensemble" else run_warmstart)(args, ws, rank, local)
    else:
        run_single(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
