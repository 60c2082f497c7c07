"""Pins of the oracle's external circuit, gap current and Fowler-Nordheim
emission (no GPU).

Sec. 2.3 drives the gap from a source through an RC circuit and emits
electrons from the cathode tip by the Fowler-Nordheim law.  The pins here do
not restate the oracle's lines; they check what physics fixes:

* charge on the anode: a charge Q landing on the anode node changes the
  capacitor's voltage by Q / C in one step (electrons lower it, ions raise it
  by their charge state, neutrals leave it alone), and the gap current is
  that charge over the electron step;
* relaxation: with nothing in the gap the anode voltage returns to the source
  voltage with the time constant RC (the explicit update is the geometric
  sequence (1 - dt/RC)^n, within about n (dt/RC)^2 / 2 of exp(-t/RC));
* FN: the constants of the elementary law come out of CODATA values here
  (A = e^3 / (8 pi h), B = 8 pi sqrt(2 m_e) / (3 e h), converted to the eV
  units of the work function), and the emitted count over many steps in a
  uniform field has the mean J(beta E) * pi r_tip^2 * dt / (e W).

Each pin is shown to catch a plausible mistake: the test compiles copies of
the oracle with one planted error each (a flipped sign, a dropped factor)
and checks that at least one pin fails on it.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synthetic

# CODATA 2018 exact and recommended values
QE = 1.602176634e-19
H = 6.62607015e-34
ME = 9.1093837015e-31
AMU = 1.66053906660e-27


def _cfg(n=16, **kw):
    c = synthetic.base_config(geometry="rz", nz=n, nr=n, dz=6e-6 / n, dr=6e-6 / n, inject_on=0,
                              field_on=2, capacity=1 << 15)
    c.update(kw)
    return c


def _oracle(cfg, lib=None):
    o = oracle.Oracle(cfg, fp64=True, lib=lib)
    g = synthetic.xs_grid()
    o.set_cross_sections({c: (g, np.zeros(g.size), 0.0) for c in range(5)})
    nn = (cfg["nz"] + 1) * (cfg["nr"] + 1)
    o.set_field(np.zeros(nn), np.zeros(nn))
    return o


def _vtol(cfg):
    """V - V0 loses the digits of V0: a few ulps of V0 bound its error."""
    return 8 * np.spacing(cfg["V0"])


def _at_anode(cfg, species, counts):
    """Particles in the last cell row before the anode, moving fast enough
    along +z to reach z = L within their first push (electrons every step,
    heavies on their sub-cycle step, which step 0 is)."""
    sp, iz, ir, pz, pr, vz = [], [], [], [], [], []
    rng = np.random.default_rng(5)
    for s, k in zip(species, counts):
        dts = cfg["dt"] * (1 if s == 0 else cfg["heavy_subcycle"])
        sp += [s] * k
        iz += [cfg["nz"] - 1] * k
        ir += list(rng.integers(0, cfg["nr"], k))
        pz += [0.5] * k
        pr += list(rng.random(k))
        vz += [0.8 * cfg["dz"] / dts] * k
    n = len(sp)
    return dict(species=np.array(sp, np.uint8), iz=np.array(iz, np.int32), ir=np.array(ir, np.int32),
                pz=np.array(pz, np.float32), pr=np.array(pr, np.float32), vz=np.array(vz, np.float32),
                vr=np.zeros(n, np.float32), vt=np.zeros(n, np.float32))


def _anode_kick(lib=None):
    """(dV, I_gap, expected Q) after one step with a mixed load reaching the anode."""
    cfg = _cfg()
    o = _oracle(cfg, lib)
    # 40 electrons, 7 Cu (neutral), 11 Cu+, 5 Cu2+ (SW label), 3 Cu2+ (DI label)
    o.load(_at_anode(cfg, [0, 1, 2, 3, 4], [40, 7, 11, 5, 3]))
    o.step(1)
    s, c = o.scalars(), o.counters()
    assert o.count() == 0
    assert c["abs_anode_e"] == 40 and c["abs_anode_Cu"] == 7 and c["abs_anode_Cu+"] == 11
    q = QE * cfg["weight"] * (-40 + 0 * 7 + 11 + 2 * 5 + 2 * 3)
    return s["V"] - cfg["V0"], s["I_gap"], q, cfg


def test_charge_on_the_anode_moves_V_by_Q_over_C():
    dV, I, q, cfg = _anode_kick()
    # q = (-40 + 27) e W < 0: net electron charge arrives, the anode voltage drops
    assert q < 0
    assert dV == pytest.approx(q / cfg["C_farad"], rel=1e-12, abs=_vtol(cfg))
    # the gap current is the charge taken from the anode node per electron step
    assert I == pytest.approx(-q / cfg["dt"], rel=1e-12)


@pytest.mark.parametrize("species,z", [(0, -1), (1, 0), (2, 1), (3, 2), (4, 2)])
def test_anode_charge_per_species(species, z):
    cfg = _cfg()
    o = _oracle(cfg)
    o.load(_at_anode(cfg, [species], [9]))
    o.step(1)
    dV = o.scalars()["V"] - cfg["V0"]
    assert dV == pytest.approx(9 * z * QE * cfg["weight"] / cfg["C_farad"], rel=1e-12, abs=_vtol(cfg))


def _relax(lib=None, nsteps=2000):
    cfg = _cfg(C_farad=1e-15)          # RC = 1 ps = 1000 electron steps
    o = _oracle(cfg, lib)
    o.load(_at_anode(cfg, [0], [200]))
    o.step(1)
    V = [o.scalars()["V"]]
    for _ in range(nsteps):
        o.step(1)
        V.append(o.scalars()["V"])
    return np.array(V), cfg


def test_rc_relaxation_to_the_source_voltage():
    V, cfg = _relax()
    V0 = cfg["V0"]
    h = cfg["dt"] / (cfg["R_ohm"] * cfg["C_farad"])
    d = V - V0
    assert d[0] < 0
    n = np.arange(len(V))
    # the explicit update is a geometric sequence with ratio 1 - dt/RC
    assert np.allclose(d, d[0] * (1 - h) ** n, rtol=1e-9, atol=0)
    # which follows exp(-t/RC) to first order in dt/RC
    dev = np.abs(d / (d[0] * np.exp(-n * h)) - 1)
    # (1 - h)^n e^(nh) = exp(-n (h^2/2 + h^3/3 + ...)) >= 1 - n h^2 (1/2 + h)
    assert np.all(dev <= n * h * h * (0.5 + h) + 1e-12)
    # two time constants in, the voltage has recovered by 1 - e^-2 of the kick
    assert abs(d[2000] / d[0] - math.exp(-2.0)) < 2e-3
    assert np.all(np.diff(V) > 0)


def fn_constants():
    """A (A eV V^-2) and B (eV^-3/2 V m^-1) of the elementary FN law from CODATA.

    J = A_SI / phi_J F^2 exp(-B_SI phi_J^(3/2) / F) with phi_J in joules,
    A_SI = e^3 / (8 pi h), B_SI = 8 pi sqrt(2 m_e) / (3 e h).  With phi in eV,
    phi_J = e phi: A = A_SI / e and B = B_SI e^(3/2)."""
    a_si = QE ** 3 / (8 * math.pi * H)
    b_si = 8 * math.pi * math.sqrt(2 * ME) / (3 * QE * H)
    return a_si / QE, b_si * QE ** 1.5


def test_fn_constants_from_codata():
    A, B = fn_constants()
    assert A == pytest.approx(1.541434e-6, rel=1e-6)
    assert B == pytest.approx(6.830890e9, rel=1e-6)


@pytest.mark.parametrize("work", [4.5, 5.1])
@pytest.mark.parametrize("F", [5e9, 1.7e10, 4e10])
def test_fn_current_against_the_law(F, work):
    A, B = fn_constants()
    J = A / work * F * F * math.exp(-B * work ** 1.5 / F)
    assert oracle.fn_current(F, work) == pytest.approx(J, rel=3e-6)


def _emission(lib=None, steps=1500):
    """Electron and neutral counts emitted in a uniform applied field (no
    self-field, collisions off) and the FN mean from the constants above."""
    cfg = _cfg(n=32, inject_on=1, tip_radius=200e-9)
    o = _oracle(cfg, lib)
    nn = (cfg["nz"] + 1) * (cfg["nr"] + 1)
    E = -cfg["V0"] / 6e-6
    o.set_field(np.full(nn, E), np.zeros(nn))
    o.step(steps)
    c = o.counters()
    A, B = fn_constants()
    F = cfg["beta"] * -E
    J = A / cfg["work_function"] * F * F * math.exp(-B * cfg["work_function"] ** 1.5 / F)
    lam = J * math.pi * cfg["tip_radius"] ** 2 * cfg["dt"] / (QE * cfg["weight"])
    ncell = math.ceil(cfg["tip_radius"] / cfg["dr"] - 1e-12)
    return c, lam * steps, ncell, steps, cfg


def test_fn_emitted_count_mean():
    c, mean_e, ncell, steps, cfg = _emission()
    assert ncell == 2
    # each tip cell draws floor(lambda + U) per step: mean lambda, variance <= 1/4
    sd = math.sqrt(ncell * steps) / 2
    assert abs(c["emitted_e"] - mean_e) < 4 * sd, (c["emitted_e"], mean_e)
    mean_n = cfg["neutral_ratio"] * mean_e
    assert abs(c["emitted_cu"] - mean_n) < 4 * sd, (c["emitted_cu"], mean_n)
    assert mean_e > 20 * sd


MUTANTS = {
    "circuit sign": ("(S->c.V0 - S->V) / S->c.R_ohm", "(S->V - S->c.V0) / S->c.R_ohm"),
    "gap current sign": ("IgapQ += -(double)ZQ[s] * QE * S->c.weight", "IgapQ += (double)ZQ[s] * QE * S->c.weight"),
    "gap current without W": ("IgapQ += -(double)ZQ[s] * QE * S->c.weight", "IgapQ += -(double)ZQ[s] * QE"),
    "FN A times phi": ("return A / work * F * F", "return A * work * F * F"),
    "FN phi^2 in the exponent": ("exp(-B * work * sqrt(work) / F)", "exp(-B * work * work / F)"),
    "FN count without W": ("J * area * S->c.dt / (QE * S->c.weight)", "J * area * S->c.dt / QE"),
    "FN area from the outer radius only": ("PI * (rhi * rhi - rlo * rlo)", "PI * rhi * rhi"),
}


def _mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pd_oracle.c")).read()
    assert src.count(old) >= 1, name          # (every copy: the serial and the OpenMP push)
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "libmut.so")
    oracle.compile_source(str(path), so, fp64=True)
    return oracle.bind(so)


def _pins_pass(lib):
    """True when every circuit and FN pin above holds for the oracle build `lib`."""
    dV, I, q, cfg = _anode_kick(lib)
    if not (math.isclose(dV, q / cfg["C_farad"], rel_tol=1e-12, abs_tol=_vtol(cfg))
            and math.isclose(I, -q / cfg["dt"], rel_tol=1e-12)):
        return False
    V, cfg = _relax(lib, nsteps=400)
    d = V - cfg["V0"]
    h = cfg["dt"] / (cfg["R_ohm"] * cfg["C_farad"])
    n = np.arange(len(V))
    if not (d[0] < 0 and np.allclose(d, d[0] * (1 - h) ** n, rtol=1e-9, atol=0)):
        return False
    A, B = fn_constants()
    for F in (5e9, 1.7e10, 4e10):
        J = A / 4.5 * F * F * math.exp(-B * 4.5 ** 1.5 / F)
        if not math.isclose(lib.or_fn_current(F, 4.5), J, rel_tol=3e-6):
            return False
    try:
        c, mean_e, ncell, steps, cfg = _emission(lib, steps=600)
    except RuntimeError:          # e.g. the capacity overflows under a 100x count
        return False
    return abs(c["emitted_e"] - mean_e) < 4 * math.sqrt(ncell * steps) / 2


def test_pins_pass_on_the_oracle(tmp_path):
    src = os.path.join(os.path.dirname(oracle.__file__), "pd_oracle.c")
    so = str(tmp_path / "libsame.so")
    oracle.compile_source(src, so, fp64=True)
    assert _pins_pass(oracle.bind(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    assert not _pins_pass(_mutant(tmp_path, name)), name
