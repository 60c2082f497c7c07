"""Long breakdown runs: the paper's setting (Sec. 2.3) stepped for up to
1e6 electron steps (1 ns at 1 fs) under CUDA graphs, with the diagnostics of
Sec. 3 sampled every few thousand steps: arc voltage and gap current, the
ionization degree and mean ion charge of Eq. (21), the cathode erosion
rate, and the Cu2+ populations by the channel that made them.

    python -m paper_2109_00214_gb300.longrun --steps 1000000 --every 10000 \\
        --out run.csv

Every step runs on the GPU; the host only reads the scalars and counters at
the sampling points.  The inputs (cross sections, sputtering yield) are the
closed-form stand-ins of `synthetic` unless the caller loads real tables
through the library's API.
"""
import argparse
import csv
import json
import math
import time

import numpy as np

import synthetic

from . import Simulation, load_library

COLS = ["step", "t_ns", "wall_s", "particles", "n_e", "n_cu", "n_cup", "n_cu2_sw", "n_cu2_di", "n_cu3", "n_cu4",
        "V", "I_gap", "gamma", "Qbar", "erosion_ug_per_C", "poisson_relres_max", "emitted_e", "emitted_cu",
        "sput_cathode", "ev_si", "ev_di", "ev_sw", "abs_cathode_e", "abs_cathode_heavy", "abs_cathode_ion_charge",
        "mass_kg", "charge_C"]

HEAVY = ("Cu", "Cu+", "Cu2+SW", "Cu2+DI", "Cu3+", "Cu4+")
CHARGE = {"Cu": 0, "Cu+": 1, "Cu2+SW": 2, "Cu2+DI": 2, "Cu3+": 3, "Cu4+": 4}


def paper_config(nz=120, nr=480, capacity=1 << 23, charge_max=4, heavy_coll=1, sputter=1, coulomb=0, seed=1):
    """The paper's breakdown setting: a 6 um gap in 50 nm cells (120 x 480
    cells, 6 x 24 um), 1 fs electron step, heavy step ten times longer,
    W = 100, 2.9 kV through 1 kOhm with 1 pF, a 200 nm tip with field
    enhancement 35, 3 % neutral flux, starting from vacuum; the collision
    extensions (charge states up to 4, heavy pairs, sputtering) on."""
    cfg, parts = synthetic.rz_breakdown(n=nz, seed=seed, capacity=capacity)
    cfg.update(nr=nr, charge_max=charge_max, heavy_coll=heavy_coll, sputter=sputter, coulomb=coulomb)
    return cfg, parts


def erosion_terms(row, weight):
    """The cathode erosion rate of a sampled row split into its ledger terms:
    net Cu mass M W (N_neutral + N_sputtered - N_heavy returned) over the net
    charge through the cathode, e W (N_e emitted - N_e returned + sum of z N
    of the ions it absorbed) (the charge ledger also counts the particles of
    the initial load that leave through the cathode).  With no returns and no
    sputtering the rate is 0.03 M / e = 19.76 ug/C; returning ions take mass
    back and add charge, so they pull it below that floor."""
    qe, mcu = 1.602176634e-19, 63.546 * 1.66053906660e-27
    mass = mcu * weight * (row["emitted_cu"] + row["sput_cathode"] - row["abs_cathode_heavy"])
    charge = qe * weight * (row["emitted_e"] - row["abs_cathode_e"] + row["abs_cathode_ion_charge"])
    floor = mcu * weight * row["emitted_cu"] / (qe * weight * row["emitted_e"]) if row["emitted_e"] else 0.0
    return dict(floor_ug_per_C=floor * 1e9, mass_kg=mass, charge_C=charge,
                from_terms_ug_per_C=mass / charge * 1e9 if charge else 0.0,
                returned_heavy=row["abs_cathode_heavy"], returned_ion_charge=row["abs_cathode_ion_charge"],
                returned_e=row["abs_cathode_e"], sputtered=row["sput_cathode"])


def run(steps, every, nz=120, nr=480, cycles=8, out=None, capacity=1 << 23, charge_max=4, heavy_coll=1,
        sputter=1, coulomb=0, seed=1, warm="extrapolate"):
    import torch
    load_library()
    cfg, parts = paper_config(nz, nr, capacity, charge_max, heavy_coll, sputter, coulomb, seed)
    sim = Simulation(cfg, synthetic.standin_cross_sections())
    E, Y = synthetic.standin_sputter_yield()
    sim.set_sputter_yield(E, Y)
    if len(parts["species"]):
        sim.load(parts)
    sim.set_warm_start(warm)           # each solve starts from the potential extrapolated in time
    sim.set_graph_mode(1, cycles)
    rows = []
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        sim.step(k)
        done += k
        sc = sim.scalars()
        c = sim.counters()
        n = list(sc["count"])
        rows.append(dict(step=done, t_ns=done * cfg["dt"] * 1e9, wall_s=time.perf_counter() - t0,
                         particles=int(sc["n_particles"]), n_e=n[0], n_cu=n[1], n_cup=n[2], n_cu2_sw=n[3],
                         n_cu2_di=n[4], n_cu3=n[5], n_cu4=n[6], V=sc["V"], I_gap=sc["I_gap"], gamma=sc["gamma"],
                         Qbar=sc["Qbar"], erosion_ug_per_C=sc["erosion"] * 1e9,
                         poisson_relres_max=sc["poisson_relres_max"], emitted_e=c["emitted_e"],
                         emitted_cu=c["emitted_cu"], sput_cathode=c["sput_cathode"], ev_si=c["ev_si"],
                         ev_di=c["ev_di"], ev_sw=c["ev_sw"], abs_cathode_e=c["abs_cathode_e"],
                         abs_cathode_heavy=sum(c[f"abs_cathode_{h}"] for h in HEAVY),
                         abs_cathode_ion_charge=sum(CHARGE[h] * c[f"abs_cathode_{h}"] for h in HEAVY),
                         mass_kg=sc["mass"], charge_C=sc["charge"]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if out:
        with open(out, "w", newline="") as f:
            w = csv.DictWriter(f, fieldnames=COLS)
            w.writeheader()
            w.writerows(rows)
    summary = dict(steps=steps, simulated_ns=steps * cfg["dt"] * 1e9, wall_s=wall,
                   steps_per_s=steps / wall, grid=[nz, nr], poisson_cycles=cycles, warm_start=warm,
                   worst_relres=max(r["poisson_relres_max"] for r in rows) if rows else None,
                   final=rows[-1] if rows else None,
                   erosion_terms=erosion_terms(rows[-1], cfg["weight"]) if rows else None)
    sim.close()
    return summary, rows


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--steps", type=int, default=1000000)
    p.add_argument("--every", type=int, default=10000)
    p.add_argument("--nz", type=int, default=120)
    p.add_argument("--nr", type=int, default=480)
    p.add_argument("--cycles", type=int, default=8, help="multigrid cycles per solve under the graph")
    p.add_argument("--warm", default="extrapolate", help="Poisson starting point: previous, cold, extrapolate")
    p.add_argument("--capacity", type=int, default=1 << 23)
    p.add_argument("--charge-max", type=int, default=4)
    p.add_argument("--no-heavy-coll", action="store_true")
    p.add_argument("--no-sputter", action="store_true")
    p.add_argument("--coulomb", action="store_true")
    p.add_argument("--out", default=None, help="CSV of the sampled diagnostics")
    a = p.parse_args()
    summary, _ = run(a.steps, a.every, a.nz, a.nr, a.cycles, a.out, a.capacity, a.charge_max,
                     0 if a.no_heavy_coll else 1, 0 if a.no_sputter else 1, 1 if a.coulomb else 0, warm=a.warm)
    print(json.dumps(summary, default=lambda x: float(x) if isinstance(x, (np.floating, np.integer)) else str(x)))


if __name__ == "__main__":
    main()
