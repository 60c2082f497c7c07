"""The long-run driver's setting is the paper's (Sec. 2.3): checked on the
host, and a few steps of it on the oracle (no GPU)."""
import pytest

import oracle
import synthetic


def test_paper_setting():
    from paper_2109_00214_gb300.longrun import paper_config
    cfg, parts = paper_config()
    assert (cfg["nz"], cfg["nr"]) == (120, 480)
    assert cfg["dz"] == pytest.approx(50e-9) and cfg["dr"] == pytest.approx(50e-9)
    assert cfg["nz"] * cfg["dz"] == pytest.approx(6e-6) and cfg["nr"] * cfg["dr"] == pytest.approx(24e-6)
    assert cfg["dt"] == 1e-15 and cfg["heavy_subcycle"] == 10 and cfg["weight"] == 100.0
    assert (cfg["V0"], cfg["R_ohm"], cfg["C_farad"]) == (2.9e3, 1e3, 1e-12)
    assert cfg["beta"] == 35.0 and 2 * cfg["tip_radius"] == pytest.approx(200e-9)
    assert cfg["neutral_ratio"] == 0.03 and cfg["geometry"] == "rz" and cfg["inject_on"] == 1
    assert len(parts["species"]) == 0                      # from vacuum


def test_paper_setting_steps_on_the_oracle(xs):
    from paper_2109_00214_gb300.longrun import paper_config
    cfg, _ = paper_config(capacity=1 << 16)
    o = oracle.Oracle(cfg, fp64=False)
    o.set_cross_sections(xs)
    E, Y = synthetic.standin_sputter_yield()
    o.set_sputter_yield(E, Y)
    o.prime()
    o.step(20)
    c = o.counters()
    assert c["emitted_e"] > 0
    assert o.scalars()["V"] == pytest.approx(2.9e3, rel=1e-3)
