"""Pins of the oracle's DSMC collision step (no GPU).

* Eq. (5)-(6): per-event momentum conservation and the energy change by the
  threshold, exactly (double build).
* Eq. (12)-(15): the ionization scheme's net balance -- charge exactly
  conserved; momentum and energy conserved except the electron created at
  the velocity V* of the excited atom (stage 2), so that per event
  dp = m_e V* and dKE = -I + m_e |V*|^2 / 2, exactly.
* Eq. (16)-(20): rectangle split v5 + v6 = v, v5 . v6 = 0.
* Eq. (7) isotropic scattering: first and second moments of the directions.
* Eq. (3)-(4): with frozen cold targets the DSMC operator reduces to the
  test-particle one, so event counts must match n_t <sigma v> dt N_e with
  <sigma v> integrated in closed form over the Maxwellian.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import synthetic

QE = 1.602176634e-19
ME = 9.1093837015e-31
MCU = 63.546 * 1.66053906660e-27
MR = ME * MCU / (ME + MCU)
TH = {0: 0.0, 1: 3.8, 2: 7.726, 3: 28.0, 4: 20.3, 7: 36.841, 8: 57.38}


@pytest.fixture(scope="module")
def o64(xs):
    cfg, _ = synthetic.rate_cell(n_e=1, n_t=1)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(xs)
    return o


def _ke(m, v):
    return 0.5 * m * float(np.dot(v, v))


@pytest.mark.parametrize("ch", [0, 1, 2, 3, 4, 7, 8])
def test_event_conservation(o64, ch):
    rng = np.random.default_rng(10 + ch)
    ok = 0
    for trial in range(400):
        ve = rng.normal(0, 6e6 if ch in (7, 8) else 4e6, 3)
        vt = rng.normal(0, 800.0, 3)
        r = o64.event(ch, ve, vt, subject=trial, step=7, sid=ch)
        if r is None:
            # below threshold: the relative energy must really be short of it
            eps = 0.5 * MR * float(np.dot(ve - vt, ve - vt)) / QE
            assert eps < TH[ch] * (1 + 1e-12)
            continue
        ok += 1
        ve2, vt2, new = r
        p0 = ME * ve + MCU * vt
        p1 = ME * ve2 + MCU * vt2 + sum(ME * e for e in new)
        ke0 = _ke(ME, ve) + _ke(MCU, vt)
        ke1 = _ke(ME, ve2) + _ke(MCU, vt2) + sum(_ke(ME, e) for e in new)
        if ch in (0, 1):
            assert not new
            assert np.allclose(p1, p0, rtol=0, atol=1e-12 * np.abs(ME * ve).max())
            assert ke1 - ke0 == pytest.approx(-TH[ch] * QE, abs=1e-11 * ke0)
        else:
            assert len(new) == (2 if ch == 3 else 1)
            vstar = vt2                      # the ion keeps the velocity of A*
            assert np.allclose(p1 - p0, ME * vstar, rtol=0, atol=1e-12 * np.abs(ME * ve).max())
            want = -TH[ch] * QE + 0.5 * ME * float(np.dot(vstar, vstar))
            assert ke1 - ke0 == pytest.approx(want, abs=1e-11 * ke0)
    assert ok > 100


def test_rectangle_split_invariants(o64):
    rng = np.random.default_rng(5)
    cos = []
    for k in range(3000):
        v = rng.normal(0, 2e6, 3)
        if k % 97 == 0:
            v[:2] = 0.0                      # v along z: phi undefined, take phi = 0
        v5, v6 = o64.rectangle_split(v, subject=k, step=3, sid=1)
        assert np.allclose(v5 + v6, v, rtol=0, atol=1e-9 * np.linalg.norm(v))
        assert abs(np.dot(v5, v6)) <= 1e-9 * np.dot(v, v)
        c = np.linalg.norm(v5) / np.linalg.norm(v)       # = cos(chi)
        assert np.dot(v5, v) == pytest.approx(c * c * np.dot(v, v), rel=1e-9, abs=1e-6)
        cos.append(c)
    cos = np.array(cos)
    # cos(chi) uniform on [0, 1): mean 1/2, variance 1/12
    assert abs(cos.mean() - 0.5) < 3 * math.sqrt(1 / 12 / len(cos))


def test_isotropic_scattering_moments(o64):
    """Elastic scattering on a resting heavy target: the post-collision
    relative-velocity direction is isotropic (Eq. (7) with isotropic I)."""
    n = 20000
    dirs = np.zeros((n, 3))
    for k in range(n):
        ve = np.array([1e6, 0.0, 0.0])
        r = o64.event(0, ve, np.zeros(3), subject=k, step=1, sid=0)
        u = r[0] - r[1]
        dirs[k] = u / np.linalg.norm(u)
    m = dirs.mean(0)
    assert np.all(np.abs(m) < 4 * math.sqrt(1 / 3 / n))
    m2 = (dirs ** 2).mean(0)
    assert np.all(np.abs(m2 - 1 / 3) < 4 * math.sqrt(4 / 45 / n))


def _maxwell_rate(ch, T_eV, xs_params):
    """<sigma v> (m^3/s) of the stand-in cross section over a Maxwellian of
    temperature T, closed form (Lotz with b = 0: sigma_max e I sqrt(8/(pi m T))
    E1(I/T); elastic: sqrt(8/(pi m)) T^-3/2 s0 [T^2 gamma(2, x0) +
    sqrt(E0) T^3/2 Gamma(3/2, x0)])."""
    m = MR
    T = T_eV * QE
    if ch == 0:
        s0, E0 = xs_params["sigma_el"], xs_params["e_el"] * QE
        x0 = E0 / T
        low = T * T * special.gammainc(2, x0) * special.gamma(2)
        high = math.sqrt(E0) * T ** 1.5 * special.gammaincc(1.5, x0) * special.gamma(1.5)
        return math.sqrt(8 / (math.pi * m)) * T ** -1.5 * s0 * (low + high)
    I = TH[ch] * QE
    smax = xs_params["peaks"][ch]
    return smax * math.e * I * math.sqrt(8 / (math.pi * m * T)) * special.exp1(I / T)


@pytest.mark.slow
def test_mcc_reduction_rates_match_closed_form(xs):
    """Frozen cold targets: expected events per channel = sum over trials of
    N_e n_t <sigma v> dt_coll.  Each trial is a fresh Maxwellian load (so the
    electron distribution does not drift), with a per-electron collision
    probability of a few percent."""
    params = dict(sigma_el=5e-20, e_el=10.0, peaks={1: 1e-20, 2: 3e-20, 3: 1e-21, 4: 1.5e-20, 7: 8e-21, 8: 5e-21})
    Te = 25.0
    n_e, n_t = 100000, 200000
    trials = 12
    counts = np.zeros(9)
    expect = np.zeros(9)
    # each pair class on its own (within one step the (e, Cu+) class sees the
    # electrons the (e, Cu) class has already scattered); the step-wise
    # classes of Cu2+ (either label) and Cu3+ with charge_max = 4
    for target, chans in ((1, (0, 1, 2, 3)), (2, (4,)), (3, (7,)), (4, (7,)), (5, (8,))):
        for tr in range(trials if target < 3 else trials // 2):
            cfg, parts = synthetic.rate_cell(n_e=n_e, n_t=n_t, Te_eV=Te, seed=100 + tr + 50 * target,
                                             depth=1e-4, coll_scale=4.0 if target < 3 else 16.0,
                                             target_species=target)
            cfg["charge_max"] = 4
            o = oracle.Oracle(cfg, fp64=True)
            o.set_cross_sections(xs)
            o.load(parts)
            o.step(1)
            c = o.counters()
            ev = [c["ev_el"], c["ev_exc"], c["ev_si"], c["ev_di"], c["ev_sw"], c["ev_cx"], c["ev_nn"],
                  c["ev_s3"], c["ev_s4"]]
            V = o.cell_volume(0)
            dtc = cfg["dt"] * cfg["coll_dt_scale"]
            nt = n_t * cfg["weight"] / V
            for ch in chans:
                counts[ch] += ev[ch]
                expect[ch] += n_e * nt * _maxwell_rate(ch, Te, params) * dtc
            assert c["ratio_viol"] == 0
    for ch in (0, 1, 2, 3, 4, 7, 8):
        sig = math.sqrt(expect[ch])
        # 3 sigma Poisson band plus 1 % for the in-step depletion of targets
        # and the few electrons that collide twice in a step
        assert abs(counts[ch] - expect[ch]) < 3 * sig + 0.01 * expect[ch], (ch, counts, expect)


def test_no_events_below_threshold(xs):
    """Electrons at 3 eV (below every inelastic threshold): only elastic events."""
    cfg, parts = synthetic.rate_cell(n_e=20000, n_t=20000, Te_eV=1.0, seed=9, depth=1e-5, coll_scale=20.0)
    v = np.sqrt(2 * 3.0 * QE / ME)
    sp = parts["species"] == 0
    d = np.random.default_rng(4).normal(size=(sp.sum(), 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    for k, key in enumerate(("vz", "vr", "vt")):
        parts[key][sp] = (v * d[:, k]).astype(np.float32)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(xs)
    o.load(parts)
    o.step(3)
    c = o.counters()
    assert c["ev_el"] > 100
    assert c["ev_exc"] == c["ev_si"] == c["ev_di"] == c["ev_sw"] == 0


@pytest.mark.parametrize("fp64", [True, False])
def test_step_conserves_charge_and_labels(xs, fp64):
    cfg, parts = synthetic.microbench(nz=16, nr=16, total=3e4, coll_scale=4000.0)
    o = oracle.Oracle(cfg, fp64=fp64)
    o.set_cross_sections(xs)
    o.load(parts)
    o.prime()
    zq = np.array([-1, 0, 1, 2, 2])
    q0 = int(zq[parts["species"]].sum())
    o.step(4)
    p = o.particles()
    c = o.counters()
    assert int(zq[p["species"]].sum()) == q0            # charge
    assert len(np.unique(p["id"])) == len(p["id"])      # ids unique
    n0 = np.bincount(parts["species"], minlength=5)
    n1 = np.bincount(p["species"], minlength=5)
    # species balance per channel (labels of Sec. 2.3)
    assert n1[3] == c["ev_sw"] and n1[4] == c["ev_di"]
    assert n1[0] - n0[0] == c["ev_si"] + c["ev_sw"] + 2 * c["ev_di"]
    assert n0[1] - n1[1] == c["ev_si"] + c["ev_di"]
    assert n1[2] - n0[2] == c["ev_si"] - c["ev_sw"]
    assert c["ev_di"] > 0 and c["ev_sw"] > 0 and c["ev_si"] > 0
    re, rh = o.rho()
    assert int(re.sum() + rh.sum()) == q0 * 2 ** 32      # fixed-point charge exact
    # DI off: no DI-labelled ions at all
    cfg2 = dict(cfg, di_on=0)
    o2 = oracle.Oracle(cfg2, fp64=fp64)
    o2.set_cross_sections(xs)
    o2.load(parts)
    o2.step(4)
    assert o2.counters()["ev_di"] == 0


def test_ncand_mean_matches_ntc_formula(xs):
    """Sum over cells of floor(x + R) has mean sum(x), x = N_e N_t W
    (sigma g)_max dt / V_c."""
    cfg, parts = synthetic.microbench(nz=32, nr=32, total=1e5, coll_scale=200.0)
    o = oracle.Oracle(cfg, fp64=True)
    o.set_cross_sections(xs)
    o.load(parts)
    sc = o.scalars()
    o.step(1)
    ncell = cfg["nz"] * cfg["nr"]
    cell = parts["iz"].astype(np.int64) * cfg["nr"] + parts["ir"]
    # counts after the first push: no field, heavies barely move, electrons a bit;
    # use the post-push state from a second oracle run for exactness
    o2 = oracle.Oracle(dict(cfg, coll_dt_scale=0.0), fp64=True)
    o2.set_cross_sections(xs)
    o2.load(parts)
    o2.step(1)
    p = o2.particles()
    cell = p["iz"].astype(np.int64) * cfg["nr"] + p["ir"]
    Ne = np.bincount(cell[p["species"] == 0], minlength=ncell)
    Ncu = np.bincount(cell[p["species"] == 1], minlength=ncell)
    Ni = np.bincount(cell[p["species"] == 2], minlength=ncell)
    V = o.cell_volume(0)
    f = cfg["weight"] * cfg["dt"] * cfg["coll_dt_scale"] / V
    mean = (Ne * Ncu).sum() * f * sc["sgmax0"] + (Ne * Ni).sum() * f * sc["sgmax1"]
    got = o.counters()["cand_total"]
    # floor(x + R) - x is uniform on (-1, 1] per cell: variance <= 1/4 per term
    assert abs(got - mean) < 4 * math.sqrt(2 * ncell / 4)


@pytest.mark.parametrize("charge_max", [2, 3, 4])
def test_stepwise_charge_states_balance(xs, charge_max):
    """The step-wise channels Cu2+ -> Cu3+ and Cu3+ -> Cu4+ (Sec. 2.3): charge
    conserved exactly, each event moves one ion up one charge state and adds
    one electron, and the channels beyond charge_max never fire."""
    cfg, parts = synthetic.microbench(nz=16, nr=16, total=3e4, coll_scale=20000.0, seed=3)
    cfg["charge_max"] = charge_max
    rng = np.random.default_rng(2)
    sp = parts["species"].copy()
    pick = rng.permutation(np.flatnonzero(sp == 2))[: int((sp == 2).sum()) // 2]
    sp[pick[0::3]] = 3
    sp[pick[1::3]] = 4
    if charge_max >= 3:
        sp[pick[2::3]] = 5
    parts = dict(parts, species=sp)
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    o.load(parts)
    o.prime()
    zq = np.array([-1, 0, 1, 2, 2, 3, 4])
    q0 = int(zq[sp].sum())
    o.step(4)
    p = o.particles()
    c = o.counters()
    assert int(zq[p["species"]].sum()) == q0
    n0 = np.bincount(sp, minlength=7)
    n1 = np.bincount(p["species"], minlength=7)
    assert n1[6] - n0[6] == c["ev_s4"]
    assert n1[5] - n0[5] == c["ev_s3"] - c["ev_s4"]
    assert (n1[3] + n1[4]) - (n0[3] + n0[4]) == c["ev_sw"] + c["ev_di"] - c["ev_s3"]
    assert n1[0] - n0[0] == c["ev_si"] + c["ev_sw"] + 2 * c["ev_di"] + c["ev_s3"] + c["ev_s4"]
    assert c["ev_s3"] == 0 if charge_max < 3 else c["ev_s3"] > 0
    assert c["ev_s4"] == 0 if charge_max < 4 else c["ev_s4"] > 0
    re, rh = o.rho()
    assert int(re.sum() + rh.sum()) == q0 * 2 ** 32
    sc = o.scalars()
    ions = n1[2:].sum()
    assert sc["Qbar"] == pytest.approx((zq[2:] * n1[2:]).sum() / ions, rel=1e-15)   # Eq. (21)
    assert sc["gamma"] == pytest.approx(ions / n1[1:].sum(), rel=1e-15)


def test_species_above_charge_max_refused(xs):
    cfg, parts = synthetic.rate_cell(n_e=10, n_t=10, target_species=5)
    o = oracle.Oracle(cfg, fp64=True)
    with pytest.raises(ValueError):
        o.load(parts)
