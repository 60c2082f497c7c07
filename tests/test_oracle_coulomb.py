"""Pins of the oracle's Coulomb collisions (the binary collision model of
Takizuka and Abe, 1977, applied to the e-e and e-ion pairs of each cell and,
on heavy steps, to its ion pairs), CPU only.

* a pair collision keeps |u| and shares the change of u by the reduced mass:
  momentum and kinetic energy are conserved exactly (FP64), on both branches
  of the rotation (u along the third axis or not);
* the deflection: tan(theta/2) = delta, delta = sqrt(var) Z with var =
  Kn / u^3 and Z the Irwin-Hall sum of twelve uniforms, so that
  E[1 - cos theta] = 2 (var m2 - var^2 m4 + var^3 m6 - ...) with the moments
  m2 = 1, m4 = 2.9, m6 = 1/21 + 13.5 of Z (from the uniform's cumulants
  1/12, -1/120, 1/252); the azimuth is uniform;
* the pairing: each electron is paired once per step with another electron
  (an odd count ends with a triple of three pairs) and, per ion species,
  the more numerous species once each: exact counts;
* a cold-ion beam: after one step the mean electron velocity has lost the
  fraction fe E[1 - cos theta] with var from the cell's ion density, W, V,
  dt and the Coulomb logarithm (the constant of the model);
* whole steps with Coulomb collisions alone conserve momentum and energy;
* ion pairs: exact counts on heavy steps and none between them, and a Cu2+
  beam through cold Cu+ slows at the model's rate with charges 2 and 1,
  m_ab = M/2 and the heavy step.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic

QE = 1.602176634e-19
ME = 9.1093837015e-31
MCU = 63.546 * 1.66053906660e-27
EPS0 = 8.8541878128e-12
MR = ME * MCU / (ME + MCU)


def omc_mean(var):
    """E[2 d^2 / (1 + d^2)], d = sqrt(var) Z, Z Irwin-Hall(12): the series in var."""
    m2, m4, m6 = 1.0, 2.9, 1.0 / 21.0 - 1.5 + 15.0
    return 2.0 * (var * m2 - var * var * m4 + var ** 3 * m6)


@pytest.fixture(scope="module")
def o64(xs):
    cfg, _ = synthetic.rate_cell(n_e=1, n_t=1)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(xs)
    return o


@pytest.mark.parametrize("fa,fb", [(0.5, 0.5), (MR / ME, MR / MCU)])
def test_pair_conserves_momentum_and_energy(o64, fa, fb):
    ma, mb = MR / fa, MR / fb                 # masses with the same reduced mass
    rng = np.random.default_rng(3)
    for trial in range(300):
        va = rng.normal(0, 2e6, 3)
        vb = rng.normal(0, 2e6 if fb == 0.5 else 1e3, 3)
        if trial % 10 == 0:
            va[:2] = vb[:2]                   # u along the third axis
        Kn = 10.0 ** rng.uniform(14, 20)
        r = o64.coulomb(va, vb, Kn, fa, fb, subject=trial, step=2, sid=9)
        assert r is not None
        va2, vb2 = r
        p0, p1 = ma * va + mb * vb, ma * va2 + mb * vb2
        assert np.allclose(p1, p0, rtol=0, atol=1e-12 * np.abs(ma * va).max() + 1e-12 * np.abs(mb * vb).max())
        e0 = 0.5 * ma * va @ va + 0.5 * mb * vb @ vb
        e1 = 0.5 * ma * va2 @ va2 + 0.5 * mb * vb2 @ vb2
        assert e1 == pytest.approx(e0, rel=1e-12)
        u0, u1 = va - vb, va2 - vb2
        assert np.linalg.norm(u1) == pytest.approx(np.linalg.norm(u0), rel=1e-12)


def test_zero_relative_velocity_is_left_alone(o64):
    v = np.array([1e5, -2e5, 3e5])
    assert o64.coulomb(v, v, 1e18, 0.5, 0.5) is None


@pytest.mark.parametrize("u,var", [(2e6, 0.01), (4e6, 0.01 / 8), (1e6, 0.004)])
def test_deflection_moments(o64, u, var):
    """var = Kn / u^3: the mean of 1 - cos(theta) follows the Irwin-Hall
    series, and the azimuth of the deflection is uniform."""
    n = 40000
    Kn = var * u ** 3
    rng = np.random.default_rng(7)
    omc = np.empty(n)
    cphi = np.empty(n)
    for k in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        va, vb = u * d, np.zeros(3)
        va2, _ = o64.coulomb(va, vb, Kn, 1.0, 0.0, subject=k, step=1, sid=3)
        c = va2 @ va / (u * u)
        omc[k] = 1.0 - c
        # azimuth about u, measured from the projection of a fixed axis
        e1 = np.cross(d, [0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.cross(d, [1.0, 0.0, 0.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(d, e1)
        w = va2 - (va2 @ d) * d
        cphi[k] = (w @ e1) / max(np.linalg.norm(w), 1e-300)
    want = omc_mean(var)
    sd = omc.std() / math.sqrt(n)
    assert abs(omc.mean() - want) < 4 * sd, (omc.mean(), want, sd)
    assert abs(cphi.mean()) < 4 / math.sqrt(2 * n)
    assert abs((cphi ** 2).mean() - 0.5) < 4 * math.sqrt(1 / 8 / n)


def test_permutation_is_a_bijection():
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 4, 5, 17, 64, 65, 1000, 4097):
        key = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
        ys = [oracle.perm_index(x, n, key) for x in range(n)]
        assert sorted(ys) == list(range(n)), n
    # different keys give different orders
    a = [oracle.perm_index(x, 100, [1, 2, 3, 4]) for x in range(100)]
    b = [oracle.perm_index(x, 100, [1, 2, 3, 5]) for x in range(100)]
    assert a != b


def _zero_xs(xs):
    return {ch: (E, np.zeros_like(s), th) for ch, (E, s, th) in xs.items()}


def test_pair_counts(xs):
    """Per step: e-e pairs N/2 (even N) or (N-3)/2 + 3 (odd N >= 3); e-ion
    pairs max(N_e, N_i) per ion species present.  The counts of the first
    step come from the load (no DSMC: zero cross sections)."""
    cfg, parts = synthetic.microbench(nz=8, nr=8, total=3e4, seed=4)
    cfg.update(coulomb=1, charge_max=3, coll_dt_scale=1.0)
    sp = parts["species"].copy()
    sp[np.flatnonzero(sp == 2)[::4]] = 3
    sp[np.flatnonzero(sp == 2)[1::4]] = 5
    parts = dict(parts, species=sp)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(_zero_xs(xs))
    o.load(parts)
    # the step's lists are those after the push: take them from a run with Coulomb off
    o2 = oracle.Oracle(dict(cfg, coulomb=0), fp64=True)
    o2.set_cross_sections(_zero_xs(xs))
    o2.load(parts)
    o2.step(1)
    p = o2.particles()
    cell = p["iz"].astype(np.int64) * cfg["nr"] + p["ir"]
    C = cfg["nz"] * cfg["nr"]
    Ne = np.bincount(cell[p["species"] == 0], minlength=C)
    ee = np.where(Ne % 2 == 0, Ne // 2, np.where(Ne >= 3, (Ne - 3) // 2 + 3, 0)).sum()
    ei = 0
    for s in (2, 3, 4, 5, 6):
        Ni = np.bincount(cell[p["species"] == s], minlength=C)
        ei += np.where((Ne > 0) & (Ni > 0), np.maximum(Ne, Ni), 0).sum()
    o.step(1)
    c = o.counters()
    assert c["coul_ee"] == ee and c["coul_ei"] == ei
    assert ee > 0 and ei > 0


def test_cold_ion_beam_loses_momentum_at_the_model_rate(xs):
    """One step of a mono-energetic electron beam through cold Cu+ (more
    electrons than ions per cell): each electron is deflected once, with
    var = Kn / v0^3, Kn = (e^2)^2 n_i lnL dt / (8 pi eps0^2 m_r^2), n_i the
    cell's ion density."""
    ncell = 64
    ne_c, ni_c = 600, 100
    v0 = 2.0e6
    lnl = 10.0
    cfg = synthetic.base_config(geometry="xy_periodic", nz=8, nr=8, dz=50e-9, dr=50e-9, depth=1e-6, dt=1e-15,
                                heavy_subcycle=1, weight=100.0, seed=5, field_on=0, inject_on=0,
                                coll_dt_scale=1.0, capacity=ncell * (ne_c + ni_c) + 1024, coulomb=1,
                                coulomb_lnl=lnl)
    rng = np.random.default_rng(2)
    cells = np.repeat(np.arange(ncell), ne_c + ni_c)
    sp = np.tile(np.r_[np.zeros(ne_c, np.uint8), np.full(ni_c, 2, np.uint8)], ncell)
    n = len(sp)
    vz = np.where(sp == 0, v0, 0.0).astype(np.float32)
    # mid-cell positions: no electron crosses a cell in one step (v0 dt = 2 nm)
    parts = dict(species=sp, iz=(cells // 8).astype(np.int32), ir=(cells % 8).astype(np.int32),
                 pz=rng.uniform(0.2, 0.8, n).astype(np.float32), pr=rng.uniform(0.2, 0.8, n).astype(np.float32),
                 vz=vz, vr=np.zeros(n, np.float32), vt=np.zeros(n, np.float32))
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(_zero_xs(xs))
    o.load(parts)
    o.step(1)
    p = o.particles()
    e = p["species"] == 0
    V = o.cell_volume(0)
    ni = ni_c * cfg["weight"] / V
    Kn = (QE * QE) ** 2 * ni * lnl * cfg["dt"] / (8 * math.pi * EPS0 ** 2 * MR ** 2)
    var = Kn / v0 ** 3
    assert 1e-3 < var < 3e-2
    fe = MR / ME
    loss = 1.0 - p["vz"][e].mean() / v0
    want = fe * omc_mean(var)
    # spread of the loss: fe (1 - cos theta) per electron, one collision each
    sd = fe * 2 * var * math.sqrt(1.9) / math.sqrt(e.sum())
    assert abs(loss - want) < 4 * sd + 1e-3 * want, (loss, want, sd)
    assert o.counters()["coul_ei"] == ncell * ne_c


def test_steps_conserve_momentum_and_energy(xs):
    cfg, parts = synthetic.microbench(nz=8, nr=8, total=2e4, seed=6)
    cfg.update(coulomb=1, coll_dt_scale=30.0)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(_zero_xs(xs))
    o.load(parts)

    def totals(p):
        m = np.where(p["species"] == 0, ME, MCU)
        v = np.stack([p["vz"], p["vr"], p["vt"]], 1)
        return (m[:, None] * v).sum(0), 0.5 * (m * (v * v).sum(1)).sum(), np.abs(m[:, None] * v).sum()

    p0, e0, s0 = totals(o.particles())
    o.step(3)
    p1, e1, _ = totals(o.particles())
    c = o.counters()
    assert c["coul_ee"] > 0 and c["coul_ei"] > 0
    assert np.all(np.abs(p1 - p0) < 1e-12 * s0)
    assert e1 == pytest.approx(e0, rel=1e-12)


def test_off_by_default(xs):
    cfg, parts = synthetic.microbench(nz=8, nr=8, total=1e4, seed=6)
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    o.load(parts)
    o.step(2)
    c = o.counters()
    assert c["coul_ee"] == 0 and c["coul_ei"] == 0


def test_ion_pairs_on_heavy_steps_only(xs):
    """Ion-ion pairs run on heavy steps: per species N/2 (even) or
    (N-3)/2 + 3 (odd) pairs, per pair of species max(N_a, N_b)."""
    cfg, parts = synthetic.microbench(nz=8, nr=8, total=3e4, seed=4)
    cfg.update(coulomb=1, charge_max=3, heavy_subcycle=10)
    sp = parts["species"].copy()
    sp[np.flatnonzero(sp == 2)[::3]] = 3
    sp[np.flatnonzero(sp == 2)[1::3]] = 5
    parts = dict(parts, species=sp)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(_zero_xs(xs))
    o.load(parts)
    o.step(1)                                 # step 0 is a heavy step: lists as loaded (heavies moved)
    c1 = o.counters()
    o2 = oracle.Oracle(dict(cfg, coulomb=0), fp64=True)
    o2.set_cross_sections(_zero_xs(xs))
    o2.load(parts)
    o2.step(1)
    p = o2.particles()
    cell = p["iz"].astype(np.int64) * cfg["nr"] + p["ir"]
    C = cfg["nz"] * cfg["nr"]
    N = {s: np.bincount(cell[p["species"] == s], minlength=C) for s in (2, 3, 4, 5, 6)}
    want = 0
    ions = (2, 3, 4, 5, 6)
    for ia, a in enumerate(ions):
        Na = N[a]
        want += np.where(Na % 2 == 0, Na // 2, np.where(Na >= 3, (Na - 3) // 2 + 3, 0)).sum()
        for b in ions[ia + 1:]:
            want += np.where((Na > 0) & (N[b] > 0), np.maximum(Na, N[b]), 0).sum()
    assert c1["coul_ii"] == want and want > 0
    o.step(5)                                 # steps 1-5: no heavy step
    assert o.counters()["coul_ii"] == c1["coul_ii"]


def test_ion_beam_through_cold_ions_at_the_model_rate(xs):
    """One heavy step of a Cu2+ beam through cold Cu+ (more beam ions than
    targets): var = (2 e^2)^2 n_Cu+ lnL dt_h / (8 pi eps0^2 (M/2)^2) / v0^3, and
    the beam's mean velocity loses the fraction E[1 - cos theta] / 2 (equal
    masses); the beam's own pairs keep its momentum."""
    ncell, nb_c, nt_c = 64, 600, 100
    lnl, W, dt, hs = 10.0, 100.0, 1e-15, 10
    V = 50e-9 * 50e-9 * 1e-6
    ni = nt_c * W / V
    Kn = (2 * QE * QE) ** 2 * ni * lnl * dt * hs / (8 * math.pi * EPS0 ** 2 * (MCU / 2) ** 2)
    v0 = (Kn / 0.01) ** (1 / 3)                  # var = 0.01
    cfg = synthetic.base_config(geometry="xy_periodic", nz=8, nr=8, dz=50e-9, dr=50e-9, depth=1e-6, dt=dt,
                                heavy_subcycle=hs, weight=W, seed=5, field_on=0, inject_on=0, coll_dt_scale=1.0,
                                capacity=ncell * (nb_c + nt_c) + 1024, coulomb=1, coulomb_lnl=lnl)
    rng = np.random.default_rng(3)
    cells = np.repeat(np.arange(ncell), nb_c + nt_c)
    sp = np.tile(np.r_[np.full(nb_c, 3, np.uint8), np.full(nt_c, 2, np.uint8)], ncell)
    n = len(sp)
    parts = dict(species=sp, iz=(cells // 8).astype(np.int32), ir=(cells % 8).astype(np.int32),
                 pz=rng.uniform(0.2, 0.8, n).astype(np.float32), pr=rng.uniform(0.2, 0.8, n).astype(np.float32),
                 vz=np.where(sp == 3, v0, 0.0).astype(np.float32), vr=np.zeros(n, np.float32),
                 vt=np.zeros(n, np.float32))
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(_zero_xs(xs))
    o.load(parts)
    o.step(1)
    p = o.particles()
    beam = p["species"] == 3
    loss = 1.0 - p["vz"][beam].mean() / float(np.float32(v0))
    var = Kn / float(np.float32(v0)) ** 3
    want = 0.5 * omc_mean(var)
    sd = 0.5 * 2 * var * math.sqrt(1.9) / math.sqrt(beam.sum())
    assert abs(loss - want) < 4 * sd + 2e-3 * want, (loss, want, sd)
