"""Precision of the FP32 state against the FP64 oracle on the small
breakdown (64 x 64 r-z cells over the 6 um gap, 500 steps of 1 fs, heavies
every 10th, self-consistent Poisson field), with double ionization on and its
twin with it off (Sec. 2.3, the two simulation sets of Sec. 3).

The library keeps particle positions and velocities in FP32 (cell-relative
positions), the oracle in FP64; both draw the same Philox numbers, so the two
runs start identical and drift apart only through rounding.  A plasma's
collective motion amplifies any difference (one particle's velocity changed
by 1e-6 in the FP64 oracle changes the spectra by step 400), so after 500
steps the FP32 run is statistically another realization of the same
physics.  The bar is the method's own statistical error:

* exact, in each run on its own: species and charge balance (every particle
  is injected, loaded or made by an event, and is present or absorbed);
* counts (events per channel, species, emitted and absorbed particles):
  |N_fp32 - N_fp64| within 2 sigma of the difference of two Poisson counts,
  2 sqrt(N_fp32 + N_fp64), plus one;
* spectra (per species and Cu2+ label, 0-500 eV in 5 eV bins) and mean
  energies: bounded loosely (L1 distance of the normalized histograms
  <= 0.25, mean energy within 35 %), and reported beside the spread of
  independent FP64 runs (other seeds; the largest pair distance).  FP64
  runs whose initial velocities differ by 1e-7 (relative) already differ
  by 10-15 % in the Cu+ mean energy after 500 steps.  The
  collective motion makes the histograms over-dispersed against Poisson
  counting, and the ions' energies follow the potential's evolution, which
  rounding perturbs more than collision noise does: an FP32 run differs from
  the FP64 one like another realization, not within the FP64 seeds' spread;
* scalars (V, I, gamma, Q, erosion) and density maps: the relative error
  is reported; V is bounded (it follows the anode charge, a count).

Two starts: from vacuum as stated (FN electrons and 3 % neutrals at the
tip; in 500 fs the first electrons cross the gap but nothing collides yet),
and the same domain seeded with a near-cathode plume of 2e4 particles (no
emission), which collides, ionizes and makes Cu2+ of both labels within the
500 steps.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

SPECIES = ["e", "Cu", "Cu+", "Cu2+SW", "Cu2+DI"]
WALLS = ("cathode", "anode", "wall")


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00214_gb300 as m
    m.load_library()
    return m


def case(kind, di):
    if kind == "vacuum":
        cfg, parts = synthetic.rz_breakdown(n=64, seed=1, di_on=di)
    else:
        cfg, parts = synthetic.rz_plume(n=64, total=2e4, seed=11, capacity=1 << 16)
        cfg.update(field_on=1, inject_on=0, di_on=di)
    cfg.update(poisson_tol=1e-10, oracle_poisson_tol=1e-12)
    return cfg, parts


def counts_of(parts):
    return np.bincount(np.asarray(parts["species"], np.int64), minlength=7)[:5]


def balance(c, n0, present):
    """Each species: loaded + emitted + made - used - absorbed = present
    (exact integers); charge the same with charge states."""
    absorbed = [sum(c[f"abs_{w}_{s}"] for w in WALLS) for s in SPECIES]
    made = np.array([
        n0[0] + c["emitted_e"] + c["ev_si"] + 2 * c["ev_di"] + c["ev_sw"],   # e: one per ionization, two per DI
        n0[1] + c["emitted_cu"] - c["ev_si"] - c["ev_di"],
        n0[2] + c["ev_si"] - c["ev_sw"],
        n0[3] + c["ev_sw"],
        n0[4] + c["ev_di"],
    ], dtype=np.int64)
    assert np.array_equal(made - np.array(absorbed), present), (made, absorbed, present)
    z = np.array([-1, 0, 1, 2, 2])
    assert int(z @ present) == int(z @ (made - np.array(absorbed)))


def within_2sigma(a, b):
    return abs(a - b) <= 2.0 * math.sqrt(a + b) + 1.0


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(b).max() if np.ndim(b) else abs(b)
    if d == 0:
        return float(np.abs(a).max()) if np.ndim(a) else abs(float(a))
    return float(np.abs(a - b).max() / d)


QE = 1.602176634e-19
MASS = [9.1093837015e-31] + [63.546 * 1.66053906660e-27] * 4


def mean_energy(p, s):
    on = p["species"] == s
    if not on.any():
        return 0.0
    v2 = p["vz"][on].astype(np.float64) ** 2 + p["vr"][on].astype(np.float64) ** 2 + \
        p["vt"][on].astype(np.float64) ** 2
    return float(0.5 * MASS[s] * v2.mean() / QE)


def spectra(sim_or_oracle):
    return [np.asarray(sim_or_oracle.energy_spectrum(s, 0.0, 500.0, 100), np.float64) for s in range(5)]


def l1(h1, h2):
    """distance of two histograms as distributions (0 equal, 2 disjoint)"""
    n1, n2 = h1.sum(), h2.sum()
    if n1 == 0 or n2 == 0:
        return 0.0 if n1 == n2 else 2.0
    return float(np.abs(h1 / n1 - h2 / n2).sum())


def run(pd, kind, di, steps=500):
    cfg, parts = case(kind, di)
    xs = synthetic.standin_cross_sections()
    sim = pd.Simulation(cfg, xs)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(xs)
    if len(parts["species"]):
        sim.load(parts)
        o.load(parts)
    o.prime()
    sim.step(steps)
    o.step(steps)
    return cfg, parts, sim, o


def oracle_seeds(cfg, parts, seeds, steps=500):
    """spectra and mean energies of FP64 oracle runs with other Philox seeds"""
    xs = synthetic.standin_cross_sections()
    out = []
    for sd in seeds:
        o = oracle.Oracle(dict(cfg, seed=sd), fp64=True)
        o.set_cross_sections(xs)
        if len(parts["species"]):
            o.load(parts)
        o.prime()
        o.step(steps)
        p = o.particles()
        out.append((spectra(o), [mean_energy(p, s) for s in range(5)]))
    return out


@pytest.mark.parametrize("kind", ["vacuum", "plume"])
@pytest.mark.parametrize("di", [1, 0])
def test_small_breakdown_fp32_against_fp64(pd, kind, di):
    cfg, parts, sim, o = run(pd, kind, di)
    n0 = counts_of(parts)
    gc, oc = sim.counters(), o.counters()
    gpart, opart = sim.particles(), o.particles()
    gn = np.bincount(gpart["species"].astype(np.int64), minlength=7)[:5]
    on = np.bincount(opart["species"].astype(np.int64), minlength=7)[:5]
    # exact in each run
    balance(gc, n0, gn)
    balance(oc, n0, on)
    if not di:
        assert gc["ev_di"] == 0 and oc["ev_di"] == 0
    report = {}
    # counts within 2 sigma
    keys = ["ev_el", "ev_exc", "ev_si", "ev_di", "ev_sw", "emitted_e", "emitted_cu"] + \
           [f"abs_{w}_{s}" for w in WALLS for s in SPECIES]
    for k in keys:
        assert within_2sigma(gc[k], oc[k]), (k, gc[k], oc[k])
        if gc[k] or oc[k]:
            report[k] = (gc[k], oc[k])
    for s, name in enumerate(SPECIES):
        assert within_2sigma(gn[s], on[s]), (name, gn[s], on[s])
        report[f"n_{name}"] = (int(gn[s]), int(on[s]))
    # spectra and mean energies against the spread of independent FP64 runs
    g_spec, o_spec = spectra(sim), spectra(o)
    g_mean = [mean_energy(gpart, s) for s in range(5)]
    o_mean = [mean_energy(opart, s) for s in range(5)]
    others = oracle_seeds(cfg, parts, [cfg["seed"] + 100 + k for k in range(3)])
    runs = [(o_spec, o_mean)] + others
    for s, name in enumerate(SPECIES):
        pair_d = [l1(runs[i][0][s], runs[j][0][s]) for i in range(len(runs)) for j in range(i + 1, len(runs))]
        pair_e = [abs(runs[i][1][s] - runs[j][1][s]) for i in range(len(runs)) for j in range(i + 1, len(runs))]
        d = l1(g_spec[s], o_spec[s])
        de = abs(g_mean[s] - o_mean[s])
        assert d <= 0.25, (name, d, pair_d)
        assert de <= 0.35 * max(o_mean[s], 1e-3), (name, g_mean[s], o_mean[s], pair_e)
        if g_spec[s].sum() + o_spec[s].sum():
            report[f"spectrum_{name}_L1"] = (round(d, 4), round(max(pair_d), 4))
            report[f"meanE_{name}_eV"] = (round(g_mean[s], 3), round(o_mean[s], 3), round(max(pair_e), 3))
    # scalars and maps: the measured FP32-vs-FP64 error
    gs, os_ = sim.scalars(), o.scalars()
    for k in ("V", "I_gap", "gamma", "Qbar", "erosion", "mass", "charge"):
        report[f"rel_{k}"] = rel(gs[k], os_[k])
    for s, name in enumerate(SPECIES):
        if gn[s] + on[s]:
            report[f"rel_map_{name}"] = rel(sim.density_map(s), o.density_map(s))
    # V follows the charge delivered to the anode, a count: FP32 enters only
    # through the step in which a particle arrives
    assert report["rel_V"] < 1e-3
    print(f"\nprecision {kind} di={di}: " + ", ".join(f"{k}={v}" for k, v in report.items()))
