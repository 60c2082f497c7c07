"""Checkpoint and resume: a simulation restored from a checkpoint continues
bit for bit as the one that wrote it; foreign or damaged files are refused."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

FIELDS = ("id", "run", "species", "iz", "ir", "pz", "pr", "vz", "vr", "vt")


@pytest.fixture(scope="module")
def pd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00214_gb300 as m
    m.load_library()
    return m


def _runs():
    out = []
    for k, (n, V) in enumerate(((32, 3.0e3), (64, 6.0e3))):
        cfg, parts = synthetic.rz_plume(n=n, total=2e4 * (k + 1), seed=40 + k)
        cfg.update(field_on=1, inject_on=1, beta=1.0, coll_dt_scale=50.0, V0=V, run=k, poisson_tol=1e-10)
        out.append((cfg, parts))
    return out


def _make(pd, runs, xs, load=True):
    ens = pd.Ensemble([c for c, _ in runs], xs)
    if load:
        for k, (_, parts) in enumerate(runs):
            ens.load_run(k, parts)
    return ens


def _sorted(g):
    order = np.lexsort((g["id"], g["run"]))
    return {k: v[order] for k, v in g.items()}


def test_resume_is_bit_identical(pd, xs, tmp_path):
    runs = _runs()
    path = str(tmp_path / "state.pdck")
    a = _make(pd, runs, xs)
    a.step(13)                       # mid heavy sub-cycle
    a.save(path)
    a.step(9)
    b = _make(pd, runs, xs, load=False)
    b.restore(path)
    assert b.run_scalars(0)["step"] == 13
    b.step(9)
    ga, gb = _sorted(a.particles()), _sorted(b.particles())
    for key in FIELDS:
        assert np.array_equal(ga[key], gb[key]), key
    for k in range(a.R):
        assert a.run_counters(k) == b.run_counters(k)
        sa, sb = a.run_scalars(k), b.run_scalars(k)
        for key in ("V", "I_gap", "charge", "mass", "poisson_relres"):
            assert sa[key] == sb[key], (k, key)
    ra, rb = a.rho(), b.rho()
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    assert np.array_equal(a.phi(), b.phi())


def test_foreign_and_damaged_files_are_refused(pd, xs, tmp_path):
    runs = _runs()
    path = tmp_path / "state.pdck"
    a = _make(pd, runs, xs)
    a.step(2)
    a.save(str(path))
    other = [(dict(c, V0=c["V0"] + 1.0), p) for c, p in runs]
    b = _make(pd, other, xs, load=False)
    with pytest.raises(pd.PdError):
        b.restore(str(path))
    cut = tmp_path / "cut.pdck"
    cut.write_bytes(path.read_bytes()[:-100])
    c = _make(pd, runs, xs, load=False)
    with pytest.raises(pd.PdError):
        c.restore(str(cut))
    junk = tmp_path / "junk.pdck"
    junk.write_bytes(b"not a checkpoint" * 8)
    with pytest.raises(pd.PdError):
        c.restore(str(junk))
    with pytest.raises(pd.PdError):
        c.restore(str(tmp_path / "missing.pdck"))


def test_rho_phi_pairs(pd, xs):
    runs = _runs()
    a = _make(pd, runs, xs)
    a.step(2)
    rho, phi = a.rho_phi()
    assert np.array_equal(phi, a.phi())
    for k, (cfg, _) in enumerate(runs):
        dm = sum(a.run_density_map(k, sp) * q for sp, q in ((0, -1), (1, 0), (2, 1), (3, 2), (4, 2)))
        r = a.run_slice(rho, k).reshape(dm.shape)
        assert np.allclose(r, 1.602176634e-19 * dm, rtol=1e-9, atol=1e-9 * np.abs(r).max())


def test_resume_with_the_extensions(pd, xs, tmp_path):
    """Charge states up to Cu4+, heavy pairs, Coulomb pairs and sputtering
    on: the restored simulation (which never saw the sputtering yield: it
    comes from the checkpoint) continues bit for bit."""
    from test_gpu_parity import _electrode_beams
    n = 32
    cfg, parts = synthetic.rz_plume(n=n, total=2e4, seed=44)
    cfg.update(field_on=1, inject_on=1, beta=1.0, coll_dt_scale=50.0, poisson_tol=1e-10, charge_max=4,
               heavy_coll=1, coulomb=1, sputter=1, heavy_subcycle=2, capacity=1 << 18)
    parts = synthetic.concat_loads([parts, _electrode_beams(n, n, 600, seed=7)])
    E, Y = synthetic.standin_sputter_yield()
    path = str(tmp_path / "ext.pdck")
    a = pd.Simulation(cfg, xs)
    a.set_sputter_yield(E, Y)
    a.load(parts)
    a.step(3)
    a.save(path)
    a.step(4)
    b = pd.Simulation(cfg, xs)
    b.restore(path)
    b.step(4)
    ga, gb = a.particles(), b.particles()
    oa, ob = np.argsort(ga["id"]), np.argsort(gb["id"])
    for key in ("id", "species", "iz", "ir", "pz", "pr", "vz", "vr", "vt"):
        assert np.array_equal(ga[key][oa], gb[key][ob]), key
    ca, cb = a.counters(), b.counters()
    assert ca == cb
    assert ca["sput_cathode"] + ca["sput_anode"] > 0 and ca["coul_ee"] > 0
