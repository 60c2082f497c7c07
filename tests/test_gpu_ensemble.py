"""GPU parity of ensembles: several independent runs of different grid sizes,
weights, seeds and gap voltages advanced together (one launch per kernel for
all runs) must each reproduce the same run simulated alone by the CPU oracle,
bit for bit; CUDA-graph stepping must give exactly the eager result; the
batched multigrid must solve every run's Poisson problem."""
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


def _runs(field_on, sizes=(32, 48, 64), volts=(2.0e3, 5.0e3, 2.9e3)):
    runs = []
    for k, (n, V) in enumerate(zip(sizes, volts)):
        cfg, parts = synthetic.rz_plume(n=n, total=1.5e4 * (k + 1), seed=10 + k)
        # with the self-consistent field the charge noise of these small loads
        # (a few 1e4 heavy-weight particles) reaches 1e11 V/m at the cathode:
        # no tip enhancement there, or Fowler-Nordheim emission runs away
        cfg.update(field_on=field_on, inject_on=1, beta=60.0 if field_on == 2 else 1.0, coll_dt_scale=50.0, V0=V,
                   run=k, poisson_tol=1e-10, oracle_poisson_tol=1e-12)
        runs.append((cfg, parts))
    return runs


def _field(cfg, seed):
    n = cfg["nz"]
    rng = np.random.default_rng(seed)
    Ez = np.full((n + 1, n + 1), -cfg["V0"] / 6e-6) * (1 + 0.3 * rng.uniform(-1, 1, (n + 1, n + 1)))
    Er = 2e8 * rng.uniform(-1, 1, (n + 1, n + 1))
    Er[:, 0] = 0
    return Ez, Er


def _ensemble(pd, runs, xs, fields=None, graph=False):
    ens = pd.Ensemble([c for c, _ in runs], xs)
    for k, (_, parts) in enumerate(runs):
        ens.load_run(k, parts)
    if fields is not None:
        Ez = np.concatenate([f[0].ravel() for f in fields])
        Er = np.concatenate([f[1].ravel() for f in fields])
        pd.pd_set_field(ens.h, Ez, Er)
    if graph:
        ens.set_graph_mode(1, 4)
    return ens


def _split(ens, g):
    out = []
    for r in range(ens.R):
        m = g["run"] == r
        sub = {k: v[m] for k, v in g.items()}
        order = np.argsort(sub["id"], kind="stable")
        out.append({k: v[order] for k, v in sub.items()})
    return out


def test_ensemble_runs_match_their_single_oracles(pd, xs):
    runs = _runs(field_on=2)
    fields = [_field(c, 3 + k) for k, (c, _) in enumerate(runs)]
    ens = _ensemble(pd, runs, xs, fields)
    steps = 12
    ens.step(steps)
    per_run = _split(ens, ens.particles())
    re, rh = ens.rho()
    for k, (cfg, parts) in enumerate(runs):
        o = oracle.Oracle(cfg, fp64=False)
        o.set_cross_sections(xs)
        o.load(parts)
        o.set_field(*fields[k])
        o.prime()
        o.step(steps)
        op = o.particles()
        g = per_run[k]
        assert len(g["id"]) == len(op["id"]), k
        for key in ("id", "species", "iz", "ir"):
            assert np.array_equal(g[key], op[key]), (k, key)
        for key in FLOATS:
            assert np.array_equal(g[key].astype(np.float64), op[key]), (k, key)
        gc, oc = ens.run_counters(k), o.counters()
        for key in oc:
            assert gc[key] == oc[key], (k, key, gc[key], oc[key])
        oe, oh = o.rho()
        assert np.array_equal(ens.run_slice(re, k), oe) and np.array_equal(ens.run_slice(rh, k), oh)
        gs, os_ = ens.run_scalars(k), o.scalars()
        assert gs["V"] == pytest.approx(os_["V"], rel=1e-12)
    assert sum(ens.run_counters(k)["emitted_e"] for k in range(ens.R)) > 0


def test_graph_stepping_equals_eager(pd, xs):
    runs = _runs(field_on=2)
    fields = [_field(c, 7 + k) for k, (c, _) in enumerate(runs)]
    a = _ensemble(pd, runs, xs, fields, graph=False)
    b = _ensemble(pd, runs, xs, fields, graph=True)
    steps = 45          # eager steps 0-9, graph replays of steps 10-39 (period 10), eager 40-44
    a.step(steps)
    b.step(steps)
    ga, gb = _split(a, a.particles()), _split(b, b.particles())
    for k in range(a.R):
        for key in ("id", "species", "iz", "ir") + FLOATS:
            assert np.array_equal(ga[k][key], gb[k][key]), (k, key)
        assert a.run_counters(k) == b.run_counters(k)
    launches = pd.pd_profile_read(b.h)
    assert sum(n for _, n in launches.values()) > 0


def test_batched_multigrid_matches_oracle_per_run(pd, xs):
    runs = _runs(field_on=1, sizes=(32, 64, 48))
    ens = _ensemble(pd, runs, xs)
    ens.step(0)                       # deposit + solve of the initial state
    phi = ens.phi()
    for k, (cfg, parts) in enumerate(runs):
        o = oracle.Oracle(cfg, fp64=True)
        o.set_cross_sections(xs)
        o.load(parts)
        o.prime()
        ophi = o.phi()
        assert np.abs(ens.run_slice(phi, k) - ophi).max() <= 1e-8 * np.abs(ophi).max(), k
        assert ens.run_scalars(k)["poisson_relres"] <= 1e-10


def test_autotuned_shapes_leave_results_unchanged(pd, xs):
    """Every tuned kernel walks its work with a grid-stride loop and writes
    order-independent results, so the autotuner's trial steps (real steps,
    under many launch shapes) must give exactly what default shapes give."""
    runs = _runs(field_on=1)
    a = _ensemble(pd, runs, xs)
    b = _ensemble(pd, runs, xs)
    chosen = b.autotune(1)
    taken = int(b.run_scalars(0)["step"])
    assert taken > 10
    assert chosen == b.tuning()
    b.set_tuning(push_blocks_per_sm=3, scatter_blocks_per_sm=5, collide_blocks_per_sm=7, mg_threads=96,
                 mg_max_blocks=9)
    b.step(3)
    a.step(taken + 3)
    ga, gb = _split(a, a.particles()), _split(b, b.particles())
    for k in range(a.R):
        for key in ("id", "species", "iz", "ir") + FLOATS:
            assert np.array_equal(ga[k][key], gb[k][key]), (k, key)
        assert a.run_counters(k) == b.run_counters(k)
        assert abs(a.run_scalars(k)["V"] - b.run_scalars(k)["V"]) <= 1e-9 * abs(a.run_scalars(k)["V"])


def test_graph_mode_reports_the_worst_residual(pd, xs):
    runs = _runs(field_on=1)
    tol = runs[0][0]["poisson_tol"]
    ens = _ensemble(pd, runs, xs)
    ens.step(10)
    ens.set_graph_mode(1, 1)                 # one V-cycle per step: short of the tolerance
    ens.step(10)
    worst = [ens.run_scalars(k)["poisson_relres_max"] for k in range(ens.R)]
    assert max(worst) > tol
    for k in range(ens.R):
        assert worst[k] >= ens.run_scalars(k)["poisson_relres"]
    ens.set_graph_mode(1, 40)                # enough cycles: every solve converges
    ens.step(10)
    for k in range(ens.R):
        assert ens.run_scalars(k)["poisson_relres_max"] <= tol


def test_ensemble_sputtering_per_run_matches_oracle(pd, xs):
    """Each run's block of the sputtering kernel takes that run's impacts:
    counts, ids and atoms equal those of the run simulated alone."""
    from test_gpu_parity import _electrode_beams
    E, Y = synthetic.standin_sputter_yield()
    runs = []
    for c, parts in _runs(field_on=2):
        c.update(sputter=1, heavy_subcycle=1)
        n = c["nz"]
        runs.append((c, synthetic.concat_loads([parts, _electrode_beams(n, c["nr"], 800, seed=n)])))
    fields = [_field(c, 3 + k) for k, (c, _) in enumerate(runs)]
    ens = _ensemble(pd, runs, xs, fields)
    pd.pd_set_sputter_yield(ens.h, E, Y)
    steps = 3
    ens.step(steps)
    per_run = _split(ens, ens.particles())
    for k, (cfg, parts) in enumerate(runs):
        o = oracle.Oracle(cfg, fp64=False)
        o.set_cross_sections(xs)
        o.set_sputter_yield(E, Y)
        o.load(parts)
        o.set_field(*fields[k])
        o.prime()
        o.step(steps)
        op = o.particles()
        g = per_run[k]
        assert len(g["id"]) == len(op["id"]), k
        for key in ("id", "species", "iz", "ir"):
            assert np.array_equal(g[key], op[key]), (k, key)
        for key in FLOATS:
            assert np.array_equal(g[key].astype(np.float64), op[key]), (k, key)
        gc, oc = ens.run_counters(k), o.counters()
        for key in oc:
            assert gc[key] == oc[key], (k, key, gc[key], oc[key])
        assert gc["sput_cathode"] > 0
