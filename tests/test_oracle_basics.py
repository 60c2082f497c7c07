"""Pins of the CPU oracle's building blocks: Philox, cross-section lookup,
push and fixed-point deposit (no GPU).  Each check compares the oracle with
something it does not contain: published vectors, closed-form trajectories,
exact invariants."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic

GOLD = os.path.join(os.path.dirname(__file__), "golden")
QE = 1.602176634e-19
ME = 9.1093837015e-31
MCU = 63.546 * 1.66053906660e-27


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_paper_energy_speed_pair():
    # Sec. 3.3: Cu at 2e4 m/s corresponds to about 133 eV (1/2 M v^2).
    pv = json.load(open(os.path.join(GOLD, "paper_values.json")))
    v = pv["cu_speed_m_s"]["value"]
    e = 0.5 * MCU * v * v / QE
    assert abs(e - pv["cu_energy_eV"]["value"]) < 1.5


def _xs_oracle(xs, fp64=True, **kw):
    cfg, _ = synthetic.rate_cell(n_e=1, n_t=1, **kw)
    o = oracle.Oracle(cfg, fp64=fp64)
    o.set_cross_sections(xs)
    return o


def test_xs_lookup_is_piecewise_linear(xs):
    o = _xs_oracle(xs)
    E = synthetic.xs_grid()
    rng = np.random.default_rng(0)
    for ch in range(5):
        s = xs[ch][1]
        # at grid points: the table value (zero below threshold)
        for k in rng.integers(0, len(E) - 1, 50):
            want = s[k] if E[k] >= xs[ch][2] else 0.0
            assert o.xs_lookup(ch, E[k]) == pytest.approx(want, rel=1e-15, abs=0)
        # between grid points: the chord (numpy interp is an independent lerp)
        for k in rng.integers(1, len(E) - 2, 50):
            e = E[k] + rng.uniform() * (E[k + 1] - E[k])
            tab = np.where(E >= xs[ch][2], s, 0.0)
            assert o.xs_lookup(ch, e) == pytest.approx(np.interp(e, E, tab), rel=1e-12, abs=1e-40)
    # outside the table: first value below, zero above
    assert o.xs_lookup(0, 1e-6) == pytest.approx(xs[0][1][0])
    assert o.xs_lookup(0, 1e6) == 0.0


def test_ntc_majorant_bounds_sigma_g(xs):
    """(sigma g)_max must bound sigma_T(eps) g(eps) everywhere (brute force on
    a dense energy sample), and not by much."""
    o = _xs_oracle(xs)
    sc = o.scalars()
    mr = ME * MCU / (ME + MCU)
    E = np.geomspace(1e-3, 3.2e4, 200001)
    g = np.sqrt(2 * E * QE / mr)
    for k, chans in ((0, (0, 1, 2, 3)), (1, (4,))):
        sT = sum(np.interp(E, synthetic.xs_grid(), np.where(synthetic.xs_grid() >= xs[c][2], xs[c][1], 0))
                 for c in chans)
        m = (sT * g).max()
        assert sc[f"sgmax{k}"] >= m
        assert sc[f"sgmax{k}"] <= m * 1.02


def _one_particle_cfg(geometry, n=64, nr=None, **kw):
    cfg = synthetic.base_config(geometry=geometry, nz=n, nr=n if nr is None else nr, inject_on=0, field_on=0,
                                heavy_subcycle=1, capacity=64, **kw)
    return cfg


def _load_one(o, sp, z, r, vz, vr, vt, dz, dr):
    iz, ir = int(z // dz), int(r // dr)
    o.load(dict(species=np.array([sp], np.uint8), iz=np.array([iz], np.int32),
                ir=np.array([ir], np.int32), pz=np.array([z / dz - iz]), pr=np.array([r / dr - ir]),
                vz=np.array([vz]), vr=np.array([vr]), vt=np.array([vt])))


def _pos(p, dz, dr):
    return (p["iz"][0] + p["pz"][0]) * dz, (p["ir"][0] + p["pr"][0]) * dr


def test_push_uniform_field_is_exact():
    """Leapfrog with v at half steps reproduces x(t) = x0 + v0 t + a t^2/2 for
    constant acceleration (v0 taken at t = -dt/2 -> v(0) = v0 + a dt/2)."""
    n = 4000
    cfg = _one_particle_cfg("xy_periodic", n=n, nr=16, dz=1e-8, dr=1e-8, depth=1e-8)
    o = oracle.Oracle(cfg, fp64=True, field_mode=2)
    Ez = np.full((n, 16), -2.0e6)
    o.set_field(Ez, np.zeros((n, 16)))
    dz = cfg["dz"]
    z0, r0, v0 = 1000.37 * dz, 7.25 * dz, 3.0e4
    _load_one(o, 0, z0, r0, v0, 0.0, 0.0, dz, dz)
    a = -QE / ME * Ez[0, 0]
    dt = cfg["dt"]
    nsteps = 50
    o.step(nsteps)
    t = nsteps * dt
    z, r = _pos(o.particles(), dz, dz)
    v_half0 = v0 + 0.5 * a * dt
    want = z0 + v_half0 * t + 0.5 * a * t * t
    assert z == pytest.approx(want, rel=1e-12)
    assert r == pytest.approx(r0, rel=1e-15)
    assert o.particles()["vz"][0] == pytest.approx(v0 + a * t, rel=1e-12)


def test_push_rz_force_free_is_straight_line():
    """Force-free r-z motion: r(t) = |(r0 + v_r t, v_theta t)|, z linear, the
    speed and the angular momentum r v_theta conserved."""
    cfg = _one_particle_cfg("rz", n=256, dz=5e-8, dr=5e-8, V0=0.0)
    o = oracle.Oracle(cfg, fp64=True, field_mode=0)
    dz = dr = cfg["dz"]
    z0, r0, vz, vr, vt = 20.5 * dz, 40.3 * dr, 1.0e5, -3.0e5, 4.0e5
    _load_one(o, 0, z0, r0, vz, vr, vt, dz, dr)
    n = 200
    o.step(n)
    t = n * cfg["dt"]
    p = o.particles()
    z, r = _pos(p, dz, dr)
    assert z == pytest.approx(z0 + vz * t, rel=1e-12)
    assert r == pytest.approx(math.hypot(r0 + vr * t, vt * t), rel=1e-12)
    sp = math.sqrt(p["vz"][0] ** 2 + p["vr"][0] ** 2 + p["vt"][0] ** 2)
    assert sp == pytest.approx(math.sqrt(vz * vz + vr * vr + vt * vt), rel=1e-13)
    assert r * p["vt"][0] == pytest.approx(r0 * vt, rel=1e-11)


def test_push_absorbs_at_electrodes_and_wall():
    cfg = _one_particle_cfg("rz", n=16, dz=5e-8, dr=5e-8, V0=0.0)
    o = oracle.Oracle(cfg, fp64=True, field_mode=0)
    d = cfg["dz"]
    _load_one(o, 0, 0.5 * d, 3 * d, -5e7, 0, 0, d, d)       # -> cathode
    _load_one(o, 2, 15.5 * d, 3 * d, 5e7, 0, 0, d, d)       # heavy -> anode
    _load_one(o, 0, 5 * d, 15.5 * d, 0, 5e7, 0, d, d)       # -> outer wall
    o.step(1)
    c = o.counters()
    assert o.count() == 0
    assert c["abs_cathode_e"] == 1 and c["abs_anode_Cu+"] == 1 and c["abs_wall_e"] == 1


def test_deposit_weights_match_eq10():
    """Fixed-point CIC weights: the four corners sum to exactly 2^32 and each
    is the bilinear shape of Eq. (10) to within the 2^-16 quantisation."""
    rng = np.random.default_rng(1)
    for _ in range(2000):
        fz, fr = rng.uniform(0, 1, 2)
        fz = float(np.float32(fz)); fr = float(np.float32(fr))
        wz, wr = oracle.deposit_weights(fz, fr)
        az, ar = 65536 - wz, 65536 - wr
        corners = [az * ar, wz * ar, az * wr, wz * wr]
        assert sum(corners) == 2 ** 32
        exact = [(1 - fz) * (1 - fr), fz * (1 - fr), (1 - fz) * fr, fz * fr]
        for c, e in zip(corners, exact):
            assert abs(c / 2 ** 32 - e) <= 2 ** -16
        assert abs(wz - fz * 65536) <= 0.5 and abs(wr - fr * 65536) <= 0.5


def test_deposit_total_charge_exact():
    cfg, parts = synthetic.microbench(nz=16, nr=16, total=2e4, coll_scale=0.0)
    o = oracle.Oracle(cfg, fp64=False)
    o.load(parts)
    o.prime()
    re, rh = o.rho()
    zq = np.array([-1, 0, 1, 2, 2])[parts["species"]]
    assert int(re.sum() + rh.sum()) == int(zq.sum()) * 2 ** 32
    assert int(re.sum()) == -int((parts["species"] == 0).sum()) * 2 ** 32


def test_verboncoeur_volumes_give_uniform_density():
    """A uniform density in r-z (particles uniform in r^2 inside each cell and
    cell counts proportional to the annulus volume) deposits to a uniform node
    density with the Verboncoeur node volumes [24] -- including the axis node
    (pi dz dr^2 / 3) and the outer node (2 pi dz dr^2 (N/2 - 1/6))."""
    n = 8
    M = 400
    cfg = _one_particle_cfg("rz", n=n, dz=5e-8, dr=5e-8, V0=0.0)
    cfg["capacity"] = 4 * M * n * n * 2
    o = oracle.Oracle(cfg, fp64=True, field_mode=0)
    iz, ir, pz, pr = [], [], [], []
    for j in range(n):
        cnt = M * (2 * j + 1)
        k = np.arange(cnt)
        rr = np.sqrt(j * j + (k + 0.5) / M)           # uniform in r^2 over [j^2, (j+1)^2]
        for i in range(n):
            zz = (np.arange(cnt) * 0.6180339887498949 + 0.5 / cnt) % 1.0
            iz.append(np.full(cnt, i)); ir.append(np.full(cnt, j))
            pz.append(zz); pr.append(rr - j)
    N = sum(len(a) for a in iz)
    o.load(dict(species=np.full(N, 2, np.uint8), iz=np.concatenate(iz).astype(np.int32),
                ir=np.concatenate(ir).astype(np.int32), pz=np.concatenate(pz),
                pr=np.concatenate(pr), vz=np.zeros(N), vr=np.zeros(N), vt=np.zeros(N)))
    dm = o.density_map(2)
    # interior axial nodes 1..n-1; every radial node including axis and wall
    inner = dm[1:n, :]
    dens = M * cfg["weight"] / (math.pi * cfg["dr"] ** 2 * cfg["dz"])  # particles per unit volume
    assert np.allclose(inner, dens, rtol=2e-3), (inner[:, :3] / dens, inner[:, -2:] / dens)
    # the plain finite-volume axis volume (pi dz dr^2/4) would be off by 4/3
    assert not np.allclose(inner[:, 0] * (1 / 3) / (1 / 4), dens, rtol=0.1)
