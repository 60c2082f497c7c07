"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs and Philox streams.

Bar (from the method's determinism rules): event counts, labels (species
codes), ids and int64 fixed-point charge bit-exact; FP32 particle state
bit-exact as well where the field is shared (the float operations are the
same, rounded one by one), which is stricter than the 1e-5 relative tolerance
allowed for FP32 state; the Poisson potential within the solve tolerance.
"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

FLOATS = ("pz", "pr", "vz", "vr", "vt")


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00214_gb300 as m
    m.load_library()
    return m


def run_pair(pd, cfg, parts, xs, steps, field=None, fp64=False):
    sim = pd.Simulation(cfg, xs)
    o = oracle.Oracle(cfg, fp64=fp64)
    o.set_cross_sections(xs)
    if len(parts["species"]):
        sim.load(parts)
        o.load(parts)
    if field is not None:
        sim.set_field(*field)
        o.set_field(*field)
    o.prime()
    sim.step(steps)
    o.step(steps)
    return sim, o


def assert_same_particles(g, op, rtol=0.0):
    order = np.argsort(g["id"], kind="stable")
    assert len(g["id"]) == len(op["id"])
    for k in ("id", "species", "iz", "ir"):
        assert np.array_equal(g[k][order], op[k]), k
    for k in FLOATS:
        a = g[k][order].astype(np.float64)
        b = op[k]
        if rtol == 0.0:
            bad = np.flatnonzero(a != b)
            assert bad.size == 0, (k, bad[:5], a[bad[:5]], b[bad[:5]])
        else:
            assert np.allclose(a, b, rtol=rtol, atol=rtol * np.abs(b).max()), k


def assert_same_counters(gc, oc, keys=None):
    for k in keys or oc:
        assert gc[k] == oc[k], (k, gc[k], oc[k])


@pytest.mark.parametrize("n_e,n_t,ncells,scale,Te", [
    (6000, 3000, 4, 3.0, 30.0),    # 1500 e / 750 Cu per cell: tables sorted by a block, ~30 candidates per cell
    (20000, 9000, 1, 0.3, 30.0),   # one cell of 29000 particles: a block's sort in the scratch buffers
    (700, 300, 2, 1.0, 30.0),      # 350 e per cell: tables sorted by the cell's warp
    (2050, 1000, 4, 3.0, 300.0),   # about 512 e per cell (both sides of the warp / block split), many movers
    (8200, 3000, 4, 1.0, 300.0),   # about 2050 e per cell (both sides of the mid-size / large block split)
    (24600, 6000, 2, 0.1, 300.0),  # about 12300 e per cell (both sides of the shared-memory limit)
    (800, 400, 4, 100.0, 300.0),   # 200 e / 100 Cu per cell, many lookups: tables of register-cached lists
    (6000, 3000, 4, 0.1, 300.0),   # 1500 e / 750 Cu per cell, about one candidate: digit-by-digit selects
    (20000, 9000, 1, 0.0006, 30.0),  # 29000 particles in one cell, about one candidate
])
def test_dense_cells_bit_exact(pd, xs, n_e, n_t, ncells, scale, Te):
    """Cells whose id lists exceed the register-cached length: the canonical
    (ascending id) pair choice must still match the oracle exactly.  Movers
    between the cells leave the lists out of id order after the first step."""
    cfg, parts = synthetic.rate_cell(n_e=n_e, n_t=n_t, Te_eV=Te, seed=5, coll_scale=scale, ncells=ncells)
    cfg.update(nz=2, nr=max(2, ncells))     # the library's grids are at least 2 x 2: a second, empty row
    sim, o = run_pair(pd, cfg, parts, xs, 3)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["cand_total"] > 0
    assert_same_particles(sim.particles(), o.particles())


@pytest.mark.parametrize("nz,nr,total,scale,steps", [
    (64, 64, 2e5, 3000.0, 4),      # stress: about one candidate per cell
    (37, 53, 6e4, 20000.0, 3),     # ragged grid, dense collisions, many spawns
    (64, 64, 2e5, 1.0, 5),         # the paper's dt: rare candidates
])
def test_microbench_bit_exact(pd, xs, nz, nr, total, scale, steps):
    cfg, parts = synthetic.microbench(nz=nz, nr=nr, total=total, coll_scale=scale, seed=11)
    sim, o = run_pair(pd, cfg, parts, xs, steps)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    if scale > 1:
        assert gc["ev_di"] > 0 and gc["ev_sw"] > 0 and gc["ev_si"] > 0
    assert_same_particles(sim.particles(), o.particles())
    ge, gh = sim.rho()
    oe, oh = o.rho()
    assert np.array_equal(ge, oe) and np.array_equal(gh, oh)
    assert gc["ratio_viol"] == 0


def test_microbench_di_off(pd, xs):
    cfg, parts = synthetic.microbench(nz=32, nr=32, total=5e4, coll_scale=5000.0, seed=5)
    cfg["di_on"] = 0
    sim, o = run_pair(pd, cfg, parts, xs, 3)
    gc = sim.counters()
    assert gc["ev_di"] == 0
    assert_same_counters(gc, o.counters())
    assert_same_particles(sim.particles(), o.particles())


@pytest.mark.parametrize("kw,steps", [
    # about 1500 Cu / 375 Cu+ per cell: block-sorted Cu tables, warp-sorted Cu+ tables
    (dict(n_e=3000, n_cu=6000, n_cup=1500, ncells=4, coll_scale=3000.0), 3),
    # one cell of 20000 Cu: the Cu table sorted by a block in the scratch buffers
    (dict(n_e=1000, n_cu=20000, n_cup=2000, ncells=1, coll_scale=100.0), 3),
    # 200 Cu per cell and many (Cu, Cu) candidates: register-cached lists,
    # candidates of one batch sharing particles
    (dict(n_e=200, n_cu=800, n_cup=200, ncells=4, coll_scale=30000.0), 3),
    # no electrons, a couple of heavy candidates per step: digit-by-digit selects
    (dict(n_e=0, n_cu=20000, n_cup=2000, ncells=1, coll_scale=0.003), 6),
    (dict(n_e=0, n_cu=6000, n_cup=1500, ncells=4, coll_scale=3.0), 4),
])
def test_heavy_pairs_bit_exact(pd, xs, kw, steps):
    """The heavy-particle pair classes (charge exchange Cu + Cu+, elastic
    Cu + Cu) beside the electron classes, on every step: the same pairs,
    acceptances and post-collision velocities as the oracle."""
    cfg, parts = synthetic.heavy_cells(**kw)
    sim, o = run_pair(pd, cfg, parts, xs, steps)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["cand_total"] > 0
    assert_same_particles(sim.particles(), o.particles())


@pytest.mark.parametrize("nz,nr,total,scale,steps", [
    (64, 64, 2e5, 3000.0, 4),
    (32, 32, 1e5, 3e5, 3),         # about a thousand candidates per cell and step
])
def test_microbench_heavy_pairs_bit_exact(pd, xs, nz, nr, total, scale, steps):
    cfg, parts = synthetic.microbench(nz=nz, nr=nr, total=total, coll_scale=scale, seed=11)
    cfg["heavy_coll"] = 1
    cfg["capacity"] = max(cfg["capacity"], 1 << 22)   # two spawn slots per electron-class candidate
    sim, o = run_pair(pd, cfg, parts, xs, steps)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["ev_cx"] > 0 and gc["ev_nn"] > 0
    assert_same_particles(sim.particles(), o.particles())
    ge, gh = sim.rho()
    oe, oh = o.rho()
    assert np.array_equal(ge, oe) and np.array_equal(gh, oh)


def _with_charge_states(parts, charge_max, seed=2):
    """Half of the Cu+ relabelled as Cu2+ (both labels) and, with charge_max
    >= 3, Cu3+: targets for the step-wise classes from the first step."""
    rng = np.random.default_rng(seed)
    sp = parts["species"].copy()
    pick = rng.permutation(np.flatnonzero(sp == 2))[: int((sp == 2).sum()) // 2]
    sp[pick[0::3]] = 3
    sp[pick[1::3]] = 4
    if charge_max >= 3:
        sp[pick[2::3]] = 5
    return dict(parts, species=sp)


@pytest.mark.parametrize("charge_max,heavy_coll,scale,steps", [
    (4, 0, 20000.0, 4),
    (3, 0, 20000.0, 3),
    (4, 1, 3000.0, 4),             # the step-wise classes before the heavy pairs of each cell
])
def test_microbench_charge_states_bit_exact(pd, xs, charge_max, heavy_coll, scale, steps):
    # hotter electrons than the default recipe, so that Cu3+ -> Cu4+ (57 eV) fires
    cfg, parts = synthetic.microbench(nz=32, nr=48, total=6e4, coll_scale=scale, seed=3, Te_range=(40.0, 120.0))
    cfg.update(charge_max=charge_max, heavy_coll=heavy_coll, capacity=max(cfg["capacity"], 1 << 21))
    parts = _with_charge_states(parts, charge_max)
    sim, o = run_pair(pd, cfg, parts, xs, steps)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["ev_s3"] > 0
    if charge_max < 4:
        assert gc["ev_s4"] == 0
    elif not heavy_coll:
        assert gc["ev_s4"] > 0
    assert_same_particles(sim.particles(), o.particles())
    ge, gh = sim.rho()
    oe, oh = o.rho()
    assert np.array_equal(ge, oe) and np.array_equal(gh, oh)
    gs, os_ = sim.scalars(), o.scalars()
    assert gs["Qbar"] == pytest.approx(os_["Qbar"], rel=1e-14)
    assert gs["gamma"] == pytest.approx(os_["gamma"], rel=1e-14)
    assert list(gs["count"]) == [int(x) for x in np.bincount(o.particles()["species"], minlength=7)]


@pytest.mark.parametrize("target,n_t,scale", [
    (3, 9000, 0.3),                # one cell of 9000 Cu2+ (SW): the list sorted by a block
    (5, 20000, 0.5),               # 20000 Cu3+: sorted in the scratch buffers
    (4, 700, 20.0),                # 700 Cu2+ (DI): the cell's warp sorts it
    (5, 6000, 0.1),                # a few candidates: digit-by-digit selects
])
def test_dense_charge_state_cells_bit_exact(pd, xs, target, n_t, scale):
    cfg, parts = synthetic.rate_cell(n_e=3000, n_t=n_t, Te_eV=60.0, seed=8, coll_scale=scale, target_species=target)
    cfg.update(nz=2, nr=2, charge_max=4)
    sim, o = run_pair(pd, cfg, parts, xs, 3)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["cand_total"] > 0
    assert_same_particles(sim.particles(), o.particles())


def test_species_above_charge_max_refused_gpu(pd, xs):
    cfg, parts = synthetic.rate_cell(n_e=10, n_t=10, target_species=5)
    cfg.update(nz=2, nr=2)
    sim = pd.Simulation(cfg, xs)
    with pytest.raises(pd.PdError):
        sim.load(parts)
        sim.synchronize()


@pytest.mark.parametrize("charge_max,heavy_coll,scale,steps,hs", [
    (2, 0, 1.0, 3, 1),
    (4, 1, 3000.0, 3, 1),          # every ion species, after the step-wise and heavy classes
    (4, 0, 1.0, 4, 2),             # ion pairs on every other step only
])
def test_microbench_coulomb_bit_exact(pd, xs, charge_max, heavy_coll, scale, steps, hs):
    cfg, parts = synthetic.microbench(nz=32, nr=48, total=6e4, coll_scale=scale, seed=5)
    cfg.update(coulomb=1, charge_max=charge_max, heavy_coll=heavy_coll, heavy_subcycle=hs,
               capacity=max(cfg["capacity"], 1 << 21))
    if charge_max > 2:
        parts = _with_charge_states(parts, charge_max)
        sp = parts["species"].copy()
        sp[np.flatnonzero(sp == 5)[::2]] = 6           # some Cu4+ as well
        parts = dict(parts, species=sp)
    sim, o = run_pair(pd, cfg, parts, xs, steps)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["coul_ee"] > 0 and gc["coul_ei"] > 0 and gc["coul_ii"] > 0
    assert_same_particles(sim.particles(), o.particles())


@pytest.mark.parametrize("n_cup,ncells", [(3000, 1), (9, 4)])
def test_ion_only_coulomb_cells_bit_exact(pd, xs, n_cup, ncells):
    """Cells without electrons: only the ion pairs collide (heavy steps)."""
    cfg, parts = synthetic.heavy_cells(n_e=0, n_cu=500, n_cup=n_cup, ncells=ncells, coll_scale=1.0, heavy_coll=0)
    cfg.update(coulomb=1)
    sim, o = run_pair(pd, cfg, parts, xs, 2)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["coul_ii"] > 0 and gc["coul_ee"] == 0
    assert_same_particles(sim.particles(), o.particles())


@pytest.mark.parametrize("n_e,n_t,ncells", [
    (20000, 9000, 1),              # 20000 electrons: rank tables in the scratch buffers
    (300, 3000, 1),                # more ions than electrons: each electron in ten rounds
    (2000, 1, 1),                  # one ion: 2000 rounds of one pair
    (701, 300, 2),                 # about 350 electrons per cell, odd counts: triples
])
def test_dense_coulomb_cells_bit_exact(pd, xs, n_e, n_t, ncells):
    cfg, parts = synthetic.rate_cell(n_e=n_e, n_t=n_t, Te_eV=5.0, seed=12, coll_scale=1.0, target_species=2,
                                     ncells=ncells)
    cfg.update(nz=2, nr=max(2, ncells), coulomb=1)
    sim, o = run_pair(pd, cfg, parts, xs, 2)
    gc, oc = sim.counters(), o.counters()
    assert_same_counters(gc, oc)
    assert gc["coul_ee"] > 0 and gc["coul_ei"] > 0
    assert_same_particles(sim.particles(), o.particles())


def _rz_field(n, V0, seed=3):
    rng = np.random.default_rng(seed)
    Ez = np.full((n + 1, n + 1), -V0 / 6e-6) * (1 + 0.3 * rng.uniform(-1, 1, (n + 1, n + 1)))
    Er = 2e8 * rng.uniform(-1, 1, (n + 1, n + 1))
    Er[:, 0] = 0
    return Ez, Er


def test_rz_external_field_with_injection_bit_exact(pd, xs):
    """r-z push with a shared external field, heavy sub-cycling (steps 0 and
    10 move heavies), FN + neutral injection, absorbing walls and circuit."""
    n = 64
    cfg, parts = synthetic.rz_plume(n=n, total=6e4, seed=2)
    cfg.update(field_on=2, inject_on=1, beta=60.0, coll_dt_scale=50.0)
    field = _rz_field(n, cfg["V0"])
    sim, o = run_pair(pd, cfg, parts, xs, 12, field=field)
    gc, oc = sim.counters(), o.counters()
    assert gc["emitted_e"] > 0 and gc["emitted_cu"] >= 0
    assert sum(gc[k] for k in gc if k.startswith("abs_")) > 0
    assert_same_counters(gc, oc)
    assert_same_particles(sim.particles(), o.particles())
    ge, gh = sim.rho()
    oe, oh = o.rho()
    assert np.array_equal(ge, oe) and np.array_equal(gh, oh)
    gs, os_ = sim.scalars(), o.scalars()
    for k in ("V", "I_gap", "gamma", "Qbar", "mass"):
        assert gs[k] == pytest.approx(os_[k], rel=1e-12, abs=1e-300), k
    assert gs["charge"] == pytest.approx(os_["charge"], rel=1e-12)


def _electrode_beams(n, nr, count, seed=21):
    """Ions of random charge state and impact energy (20 eV .. 3 keV) one step
    from the cathode or the anode, moving onto it, with some electrons and
    neutrals doing the same."""
    rng = np.random.default_rng(seed)
    QE, MCU, ME = 1.602176634e-19, 63.546 * 1.66053906660e-27, 9.1093837015e-31
    sp = rng.choice(np.array([0, 1, 2, 3, 4], np.uint8), count, p=[0.1, 0.1, 0.5, 0.2, 0.1])
    E = 10 ** rng.uniform(np.log10(20.0), np.log10(3000.0), count)
    v = np.sqrt(2 * E * QE / np.where(sp == 0, ME, MCU))
    cat = rng.uniform(size=count) < 0.6
    return dict(species=sp, iz=np.where(cat, 0, n - 1).astype(np.int32),
                ir=rng.integers(0, nr, count).astype(np.int32),
                pz=np.where(cat, 1e-6, 1 - 1e-6).astype(np.float32), pr=rng.uniform(0, 1, count).astype(np.float32),
                vz=np.where(cat, -v, v).astype(np.float32),
                vr=(0.1 * v * rng.standard_normal(count)).astype(np.float32),
                vt=(0.1 * v * rng.standard_normal(count)).astype(np.float32))


@pytest.mark.parametrize("heavy_subcycle", [1, 10])
def test_rz_sputtering_bit_exact(pd, xs, heavy_subcycle):
    """Ions arriving at either electrode sputter Cu atoms (stand-in yield):
    the same counts, ids, positions and velocities as the oracle."""
    n = 64
    cfg, parts = synthetic.rz_plume(n=n, total=3e4, seed=4)
    cfg.update(field_on=2, inject_on=1, beta=60.0, coll_dt_scale=50.0, sputter=1, heavy_subcycle=heavy_subcycle)
    parts = synthetic.concat_loads([parts, _electrode_beams(n, n, 3000)])
    E, Y = synthetic.standin_sputter_yield()
    sim = pd.Simulation(cfg, xs)
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    sim.set_sputter_yield(E, Y)
    o.set_sputter_yield(E, Y)
    sim.load(parts)
    o.load(parts)
    field = _rz_field(n, cfg["V0"])
    sim.set_field(*field)
    o.set_field(*field)
    o.prime()
    sim.step(3)
    o.step(3)
    gc, oc = sim.counters(), o.counters()
    assert gc["sput_cathode"] > 0 and gc["sput_anode"] > 0
    assert_same_counters(gc, oc)
    assert_same_particles(sim.particles(), o.particles())
    gs, os_ = sim.scalars(), o.scalars()
    assert gs["mass"] == pytest.approx(os_["mass"], rel=1e-12)


def test_sputter_queue_overflow_is_reported(pd, xs):
    """More ion impacts in a step than the impact queue holds (4096 with this
    capacity): the step reports a capacity error instead of writing past it."""
    n = 64
    cfg, _ = synthetic.rz_plume(n=n, total=2e3, seed=4)
    cfg.update(field_on=2, inject_on=0, sputter=1, heavy_subcycle=1, capacity=60000)
    rng = np.random.default_rng(5)
    m = 6000
    QE, MCU = 1.602176634e-19, 63.546 * 1.66053906660e-27
    v = np.sqrt(2 * 500.0 * QE / MCU)
    beam = dict(species=np.full(m, 2, np.uint8), iz=np.zeros(m, np.int32), ir=rng.integers(0, n, m).astype(np.int32),
                pz=np.full(m, 1e-6, np.float32), pr=rng.uniform(0, 1, m).astype(np.float32),
                vz=np.full(m, -v, np.float32), vr=np.zeros(m, np.float32), vt=np.zeros(m, np.float32))
    sim = pd.Simulation(cfg, xs)
    E = synthetic.xs_grid()
    sim.set_sputter_yield(E, np.full_like(E, 2.0))
    sim.load(beam)
    sim.set_field(*_rz_field(n, cfg["V0"]))
    sim.step(1)
    with pytest.raises(pd.PdError, match="CAPACITY"):
        sim.synchronize()


@pytest.mark.parametrize("n,nr", [
    (64, 64),      # coarsest level 8 x 8 cells: solved by its stored inverse
    (96, 96),      # 6 x 6
    (64, 320),     # R = 5 L: coarsest 8 x 40 cells, 287 unknowns: Gauss-Seidel sweeps
    (32, 32),      # every level in the one-block tail, the correction added to phi there
    (16, 48),      # two levels, both in the tail
    (120, 480),    # the paper's domain (Sec. 2.3): 6 x 24 um in 50 nm cells
])
def test_rz_poisson_matches_oracle(pd, xs, n, nr):
    """Self-consistent field: multigrid (GPU) vs conjugate gradients (CPU) on
    the same fixed-point charge, to the solve tolerance."""
    cfg, parts = synthetic.rz_plume(n=n, total=8e4, seed=4)
    cfg.update(nr=nr, field_on=1, inject_on=0, poisson_tol=1e-10, oracle_poisson_tol=1e-12)
    sim, o = run_pair(pd, cfg, parts, xs, 0)
    sim.step(0)
    gphi, ophi = sim.phi(), o.phi()
    scale = np.abs(ophi).max()
    assert np.abs(gphi - ophi).max() <= 1e-8 * scale
    gs = sim.scalars()
    assert gs["poisson_relres"] <= 1e-10
    gEz, gEr = sim.field()
    oEz, oEr = o.field()
    assert np.allclose(gEz, oEz, rtol=1e-6, atol=1e-6 * np.abs(oEz).max())
    assert np.allclose(gEr, oEr, rtol=1e-6, atol=1e-6 * np.abs(oEz).max())


@pytest.mark.parametrize("n,nr", [(64, 64), (120, 480)])
def test_rz_self_consistent_steps_track_oracle(pd, xs, n, nr):
    """A few self-consistent steps: the two field solves agree to ~1e-9, so
    particle states agree to FP32 rounding and the counters stay equal.  The
    second case is the paper's domain, 120 x 480 cells of 50 nm (Sec. 2.3)."""
    cfg, parts = synthetic.rz_plume(n=n, total=3e4, seed=6)
    cfg.update(nr=nr, field_on=1, inject_on=1, poisson_tol=1e-10, oracle_poisson_tol=1e-12)
    sim, o = run_pair(pd, cfg, parts, xs, 5)
    gc, oc = sim.counters(), o.counters()
    for k in ("ev_el", "ev_exc", "ev_si", "ev_di", "ev_sw", "emitted_e", "emitted_cu"):
        assert abs(gc[k] - oc[k]) <= max(2, 0.01 * oc[k]), k
    g, op = sim.particles(), o.particles()
    assert abs(len(g["id"]) - len(op["id"])) <= max(4, 0.001 * len(op["id"]))


def test_empty_and_capacity(pd, xs):
    cfg, parts = synthetic.microbench(nz=16, nr=16, total=2e3, seed=1)
    sim = pd.Simulation(dict(cfg, capacity=4096), xs)
    sim.step(3)                                   # empty domain steps fine
    assert sim.counters()["cand_total"] == 0
    small = dict(cfg, capacity=100)
    sim2 = pd.Simulation(small, xs)
    with pytest.raises(pd.PdError):
        sim2.load(parts)                          # more particles than slots
    # a capacity that the spawns overrun is reported, not written past
    cfg3, parts3 = synthetic.microbench(nz=16, nr=16, total=3e3, coll_scale=2e5, seed=2)
    sim3 = pd.Simulation(dict(cfg3, capacity=len(parts3["species"]) + 8), xs)
    sim3.load(parts3)
    sim3.step(2)
    with pytest.raises(pd.PdError, match="CAPACITY"):
        sim3.synchronize()


def test_species_diagnostics_match_oracle(pd, xs):
    n = 32
    cfg, parts = synthetic.rz_plume(n=n, total=2e4, seed=9)
    cfg.update(field_on=0, inject_on=0, coll_dt_scale=200.0)
    sim, o = run_pair(pd, cfg, parts, xs, 3)
    for sp in (0, 1, 2, 3, 4):
        assert np.array_equal(sim.energy_spectrum(sp, 0, 200, 40), o.energy_spectrum(sp, 0, 200, 40))
        assert np.allclose(sim.density_map(sp), o.density_map(sp), rtol=1e-12, atol=0)
    gs, os_ = sim.scalars(), o.scalars()
    assert gs["gamma"] == pytest.approx(os_["gamma"], rel=1e-14)
    assert gs["Qbar"] == pytest.approx(os_["Qbar"], rel=1e-14)
