"""The movers-only sort on grids with more bins than particles, where the
minimum slack of every layout (three slots a bin, and the rounding up) is
most of the slots: re-layouts and borrowing must keep every particle inside
the bin of its cell, the bins disjoint and inside the slot arrays, and the
steps bit-exact against the oracle (which has no sort: it owns no layout)."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

FLOATS = ("pz", "pr", "vz", "vr", "vt")
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


def check_bins(sim, ncell):
    """Every live particle below the tail lies in [start, start + count) of a
    bin of its own cell; the bins' occupied ranges are disjoint."""
    start, count = sim.bins()
    nb = len(count)
    s0 = start[:nb].astype(np.int64)
    c0 = count.astype(np.int64)
    order = np.lexsort((c0, s0))                 # equal starts: the occupied bin last
    ss, cc = s0[order], c0[order]
    occ = cc > 0
    ends = ss[occ] + cc[occ]
    assert np.all(ends[:-1] <= ss[occ][1:]), "occupied bin ranges overlap"
    p = sim.particles(live_only=False)
    tail = int(ends.max()) if len(ends) else 0
    slot = np.arange(len(p["species"]), dtype=np.int64)
    live = (p["species"] != 255) & (slot < tail)
    k = np.searchsorted(ss, slot[live], side="right") - 1
    b = order[k]
    assert np.all(slot[live] < s0[b] + c0[b]), "a particle outside every bin"
    cell = p["iz"][live].astype(np.int64) * sim.cfg_dict["nr"] + p["ir"][live]
    assert np.array_equal(b % ncell, cell), "a particle in another cell's bin"
    return tail


def test_sparse_ensemble_run_layouts_fit(pd, xs):
    """Run 3 of the ensemble recipe's first seed (256 x 256 r-z cells, about
    1.3e5 particles, capacity 1.25 N + 65536, self-consistent field): 262 144
    heavy bins for about 6e4 heavy particles.  Forty steps with re-layouts:
    no error, bins consistent, species balance exact."""
    cfg, parts = synthetic.ensemble_breakdown(seeds=[1])[3]
    assert cfg["nz"] == 256
    sim = pd.Simulation(cfg, xs)
    sim.set_warm_start("extrapolate")
    sim.load(parts)
    n0 = np.bincount(parts["species"].astype(np.int64), minlength=7)[:5]
    for _ in range(4):
        sim.step(10)
        sim.synchronize()
        check_bins(sim, cfg["nz"] * cfg["nr"])
    st = sim.sort_stats()
    assert st["faults"] == 0
    assert st["relayouts"] >= 2, st
    c = sim.counters()
    g = sim.particles()
    gn = np.bincount(g["species"].astype(np.int64), minlength=7)[:5]
    absorbed = np.array([sum(c[f"abs_{w}_{s}"] for w in WALLS) for s in SPECIES])
    made = np.array([n0[0] + c["emitted_e"] + c["ev_si"] + 2 * c["ev_di"] + c["ev_sw"],
                     n0[1] + c["emitted_cu"] - c["ev_si"] - c["ev_di"],
                     n0[2] + c["ev_si"] - c["ev_sw"],
                     n0[3] + c["ev_sw"],
                     n0[4] + c["ev_di"]])
    assert np.array_equal(made - absorbed, gn)


@pytest.mark.parametrize("n,min_relayouts", [
    (128, 1),      # 1.2 particles a cell: bins borrow from their empty neighbours
    (48, 2),       # 8.7 a cell: borrowing falls short and the bins are laid out anew
])
def test_hot_heavies_bit_exact(pd, xs, n, min_relayouts):
    """n x n Cartesian cells, 2e4 particles, heavies hot enough to cross
    about a cell a step (2e13 K: 5e7 m/s, a 50 nm cell in a 1 fs step; the
    sort does not care that no copper is that hot), and a capacity of
    25 000: every step moves most heavy
    particles between bins of little slack, so bins borrow and the layout is
    redone; the particles must match the oracle bit for bit."""
    cfg, parts = synthetic.microbench(nz=n, nr=n, total=2e4, seed=7, T_heavy=2e13)
    cfg.update(capacity=25000)
    sim = pd.Simulation(cfg, xs)
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    sim.load(parts)
    o.load(parts)
    o.prime()
    for _ in range(3):
        sim.step(8)
        o.step(8)
        sim.synchronize()
        check_bins(sim, n * n)
    st = sim.sort_stats()
    assert st["faults"] == 0
    assert st["relayouts"] >= min_relayouts, st
    gc, oc = sim.counters(), o.counters()
    for k in oc:
        assert gc[k] == oc[k], (k, gc[k], oc[k])
    g, op = sim.particles(), o.particles()
    order = np.argsort(g["id"], kind="stable")
    assert len(g["id"]) == len(op["id"])
    for k in ("id", "species", "iz", "ir"):
        assert np.array_equal(g[k][order], op[k]), k
    for k in FLOATS:
        assert np.array_equal(g[k][order].astype(np.float64), op[k]), k
