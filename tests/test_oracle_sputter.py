"""Pins of the oracle's ion-impact sputtering (Sec. 2.3: energetic ions
arriving at the electrodes sputter neutrals into the gap; the yield is an
input table, the paper's Yamamura-Tawara data not being available), CPU only.

* the count per impact is floor(Y + R): its mean is Y exactly, for a constant
  yield and for a yield linear in the impact energy;
* sputtered atoms start on the electrode surface at the impact radius, move
  into the gap, and follow the effusive flux at sputter_T (mean normal and
  transverse speeds sqrt(pi/2) sqrt(kT/M), isotropic azimuth);
* their ids follow the run's ids in the order of the ions' ids;
* electrons and neutrals arriving at the electrodes sputter nothing, nor
  does anything with sputtering off;
* the cathode mass ledger counts sputtered atoms as mass leaving it.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic

QE = 1.602176634e-19
KB = 1.380649e-23
MCU = 63.546 * 1.66053906660e-27
ME = 9.1093837015e-31


def beam(n, E0, toward="cathode", species=2, seed=1, nz=8, nr=8):
    """n particles of one species one step from an electrode, all with impact
    energy E0 (eV) at normal incidence."""
    rng = np.random.default_rng(seed)
    m = ME if species == 0 else MCU
    v0 = math.sqrt(2 * E0 * QE / m)
    cat = toward == "cathode"
    return dict(species=np.full(n, species, np.uint8),
                iz=np.full(n, 0 if cat else nz - 1, np.int32),
                ir=rng.integers(0, nr, n).astype(np.int32),
                pz=np.full(n, 1e-6 if cat else 1 - 1e-6, np.float32),
                pr=rng.uniform(0, 1, n).astype(np.float32),
                vz=np.full(n, -v0 if cat else v0, np.float32),
                vr=np.zeros(n, np.float32), vt=np.zeros(n, np.float32))


def make(xs, Y, parts, sputter=1, T=23209.0, fp64=True):
    cfg = synthetic.base_config(geometry="rz", nz=8, nr=8, dz=50e-9, dr=50e-9, dt=1e-15, heavy_subcycle=1,
                                weight=100.0, seed=3, field_on=0, inject_on=0, coll_dt_scale=1.0,
                                capacity=len(parts["species"]) * 8 + 1024, sputter=sputter, sputter_T=T)
    o = oracle.Oracle(cfg, fp64=fp64)
    o.set_cross_sections(xs)
    E = synthetic.xs_grid()
    o.set_sputter_yield(E, Y(E))
    o.load(parts)
    return o, cfg


@pytest.mark.parametrize("Y,E0,want", [
    (lambda E: np.full_like(E, 1.7), 500.0, 1.7),
    (lambda E: 0.004 * E, 300.0, 1.2),
    (lambda E: np.full_like(E, 0.35), 2000.0, 0.35),
])
def test_mean_count_is_the_yield(xs, Y, E0, want):
    n = 20000
    o, _ = make(xs, Y, beam(n, E0))
    o.step(1)
    c = o.counters()
    assert c["abs_cathode_Cu+"] == n
    frac = want - math.floor(want)
    sd = math.sqrt(frac * (1 - frac) / n)
    assert abs(c["sput_cathode"] / n - want) < 4 * sd + 1e-12
    assert c["sput_anode"] == 0


@pytest.mark.parametrize("toward", ["cathode", "anode"])
def test_sputtered_atoms_effusive_from_the_impact_point(xs, toward):
    n, T = 20000, 23209.0
    parts = beam(n, 800.0, toward=toward)
    o, cfg = make(xs, lambda E: np.full_like(E, 2.0), parts, T=T)
    o.step(1)
    p = o.particles()
    cu = p["species"] == 1
    assert cu.sum() == 2 * n
    vth = math.sqrt(KB * T / MCU)
    vn = p["vz"][cu] if toward == "cathode" else -p["vz"][cu]
    assert np.all(vn >= 0)
    mean_rayleigh = vth * math.sqrt(math.pi / 2)
    sd = vth * math.sqrt((4 - math.pi) / 2) / math.sqrt(cu.sum())
    assert abs(vn.mean() - mean_rayleigh) < 4 * sd
    s = np.hypot(p["vr"][cu], p["vt"][cu])
    assert abs(s.mean() - mean_rayleigh) < 4 * sd
    phi = np.arctan2(p["vt"][cu], p["vr"][cu])
    assert abs(np.cos(phi).mean()) < 4 / math.sqrt(2 * cu.sum())
    # on the electrode surface, at the radius of an impact
    if toward == "cathode":
        assert np.all(p["iz"][cu] == 0) and np.all(p["pz"][cu] == 0.0)
    else:
        assert np.all(p["iz"][cu] == cfg["nz"] - 1) and np.all(p["pz"][cu] >= 1 - 1e-15)
    impact = set(zip(parts["ir"].tolist(), parts["pr"].astype(np.float64).tolist()))
    got = set(zip(p["ir"][cu].tolist(), p["pr"][cu].tolist()))
    assert got <= impact


def test_ids_follow_the_ions_ids(xs):
    n = 500
    parts = beam(n, 800.0, seed=4)
    o, _ = make(xs, lambda E: np.full_like(E, 2.0), parts)
    o.step(1)
    p = o.particles()
    cu = p["species"] == 1
    ids = np.sort(p["id"][cu])
    assert np.array_equal(ids, np.arange(n, n + 2 * n))        # the ions held ids 0..n-1
    # the two atoms of ion k (id k) are ids n + 2k, n + 2k + 1: same impact radius
    order = np.argsort(p["id"][cu])
    pr = p["pr"][cu][order]
    assert np.array_equal(pr[0::2], pr[1::2])
    assert np.allclose(pr[0::2], parts["pr"].astype(np.float64))


def test_electrons_and_neutrals_do_not_sputter(xs):
    parts = synthetic.concat_loads([beam(2000, 800.0, species=0), beam(2000, 800.0, species=1, seed=2)])
    o, _ = make(xs, lambda E: np.full_like(E, 2.0), parts)
    o.step(1)
    c = o.counters()
    assert c["abs_cathode_e"] == 2000 and c["abs_cathode_Cu"] == 2000
    assert c["sput_cathode"] == 0


def test_off_changes_nothing(xs):
    parts = beam(3000, 800.0)
    o, _ = make(xs, lambda E: np.full_like(E, 2.0), parts, sputter=0)
    o.step(1)
    assert o.counters()["sput_cathode"] == 0
    assert (o.particles()["species"] == 1).sum() == 0


def test_cathode_mass_ledger_counts_sputtered_atoms(xs):
    n = 4000
    o, cfg = make(xs, lambda E: np.full_like(E, 1.5), beam(n, 600.0))
    o.step(1)
    c = o.counters()
    sc = o.scalars()
    want = MCU * cfg["weight"] * (c["emitted_cu"] + c["sput_cathode"] - n)
    assert sc["mass"] == pytest.approx(want, rel=1e-12)
    assert c["sput_cathode"] > n          # more atoms leave than ions arrive: net erosion
