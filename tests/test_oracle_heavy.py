"""Oracle pins of the heavy-particle pair classes (resonant charge exchange
Cu+ + Cu and elastic Cu + Cu, the collisions besides ionization that the
paper's Sec. 2.3 lists), CPU only.

* rates: for Maxwellian Cu and Cu+ at T with a constant cross section, the
  number of events per heavy step is N_a N_b W sigma <g> dt_coll / V
  (N (N - 1) / 2 pairs for Cu + Cu), <g> = sqrt(16 k T / (pi M)) for two
  Maxwellians of mass M (the relative velocity is Maxwellian with mass M/2);
* charge exchange only swaps velocities: the multiset of heavy velocity
  vectors is unchanged, exactly;
* the elastic collisions conserve momentum and kinetic energy (FP64);
* with the classes off nothing changes.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic
from synthetic.workloads import _KB, _MCU

pytestmark = pytest.mark.filterwarnings("ignore")

T = 2000.0
D = 50e-9
DEPTH = 1e-6


def heavy_cell(n_cu, n_cup, seed=7):
    rng = np.random.default_rng(seed)
    vs = math.sqrt(_KB * T / _MCU)
    n = n_cu + n_cup
    parts = {
        "species": np.r_[np.full(n_cu, 1, np.uint8), np.full(n_cup, 2, np.uint8)],
        "iz": np.zeros(n, np.int32), "ir": np.zeros(n, np.int32),
        "pz": rng.uniform(0, 1, n).astype(np.float32), "pr": rng.uniform(0, 1, n).astype(np.float32),
        "vz": (rng.standard_normal(n) * vs).astype(np.float32),
        "vr": (rng.standard_normal(n) * vs).astype(np.float32),
        "vt": (rng.standard_normal(n) * vs).astype(np.float32),
    }
    return parts


def xs_flat(s_cx, s_nn, e_max=10.0):
    """The stand-in tables with constant heavy cross sections up to e_max eV
    (thermal relative energies are ~0.2 eV at 2000 K)."""
    xs = synthetic.standin_cross_sections()
    E = xs[5][0]
    xs[5] = (E, np.where(E <= e_max, s_cx, 0.0), 0.0)
    xs[6] = (E, np.where(E <= e_max, s_nn, 0.0), 0.0)
    return xs


def make(parts, xs, heavy_coll=1, coll_scale=1000.0, fp64=True, seed=3):
    cfg = synthetic.base_config(geometry="xy_periodic", nz=1, nr=1, dz=D, dr=D, depth=DEPTH, dt=1e-15,
                                heavy_subcycle=10, weight=100.0, seed=seed, field_on=0, inject_on=0,
                                coll_dt_scale=coll_scale, capacity=len(parts["species"]) + 1024,
                                heavy_coll=heavy_coll)
    o = oracle.Oracle(cfg, fp64=fp64)
    o.set_cross_sections(xs)
    o.load(parts)
    o.prime()
    return o, cfg


def expected_per_heavy_step(pairs, sigma, cfg):
    g_mean = math.sqrt(16.0 * _KB * T / (math.pi * _MCU))
    dt_coll = cfg["dt"] * cfg["heavy_subcycle"] * cfg["coll_dt_scale"]
    return pairs * cfg["weight"] * sigma * g_mean * dt_coll / (D * D * DEPTH)


@pytest.mark.parametrize("kind", ["cx", "nn"])
def test_heavy_rates(kind):
    n_cu, n_cup = 3000, 1500
    s = 6e-19 if kind == "cx" else 2.1e-19
    xs = xs_flat(s if kind == "cx" else 0.0, s if kind == "nn" else 0.0)
    o, cfg = make(heavy_cell(n_cu, n_cup), xs)
    heavy_steps = 8
    o.step(10 * heavy_steps)
    c = o.counters()
    pairs = n_cu * n_cup if kind == "cx" else 0.5 * n_cu * (n_cu - 1)
    mu = heavy_steps * expected_per_heavy_step(pairs, s, cfg)
    got = c["ev_" + kind]
    assert mu > 500
    assert abs(got - mu) < 4.0 * math.sqrt(mu) + 0.01 * mu, (got, mu)
    assert c["ev_" + ("nn" if kind == "cx" else "cx")] == 0
    assert c["ratio_viol"] == 0


def test_charge_exchange_only_permutes_velocities():
    parts = heavy_cell(800, 600)
    o, _ = make(parts, xs_flat(6e-19, 0.0), fp64=False)
    before = np.stack([parts["vz"], parts["vr"], parts["vt"]], 1)
    o.step(40)
    assert o.counters()["ev_cx"] > 100
    p = o.particles()
    after = np.stack([p["vz"], p["vr"], p["vt"]], 1).astype(np.float32)
    key = lambda a: a[np.lexsort(a.T[::-1])]
    assert np.array_equal(key(before), key(after))
    # the species (and so the charge) stay with their slots
    assert int(np.sum(p["species"] == 2)) == 600


def test_cu_elastic_conserves_momentum_and_energy():
    parts = heavy_cell(1500, 0)
    o, _ = make(parts, xs_flat(0.0, 2.1e-19))
    v0 = np.stack([parts["vz"], parts["vr"], parts["vt"]], 1).astype(np.float64)
    o.step(40)
    assert o.counters()["ev_nn"] > 100
    p = o.particles()
    v1 = np.stack([p["vz"], p["vr"], p["vt"]], 1)
    assert np.allclose(v1.sum(0), v0.sum(0), rtol=0, atol=1e-9 * np.abs(v0).sum())
    e0, e1 = (v0 ** 2).sum(), (v1 ** 2).sum()
    assert abs(e1 - e0) <= 1e-12 * e0
    assert not np.array_equal(np.sort(v0[:, 0]), np.sort(v1[:, 0]))   # velocities did change


def test_heavy_classes_off_by_default():
    o, _ = make(heavy_cell(800, 600), xs_flat(6e-19, 2.1e-19), heavy_coll=0)
    o.step(20)
    c = o.counters()
    assert c["ev_cx"] == 0 and c["ev_nn"] == 0 and c["cand_total"] == 0
