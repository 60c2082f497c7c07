"""Host-side checks of the C ABI (no GPU): the library builds, loads and
exports every function include/pd.h declares; configuration validation and
workspace sizing work without a device."""
import ctypes as C
import os
import re

import pytest

import paper_2109_00214_gb300 as pd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = pd.load_library()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(pd.EXPORTED)


def test_config_default_is_the_papers():
    c = pd.pd_config_default()
    assert c.struct_size == C.sizeof(pd.PdConfig)
    assert c.dt == 1e-15 and c.heavy_subcycle == 10 and c.weight == 100.0
    assert c.V0 == 2.9e3 and c.R_ohm == 1e3 and c.C_farad == 1e-12
    assert c.beta == 35.0 and c.tip_radius == 100e-9 and c.neutral_ratio == 0.03


def test_workspace_size_and_validation():
    import synthetic
    cfg, _ = synthetic.microbench(nz=64, nr=64, total=1e5)
    c = pd.config_from_dict(cfg)
    n = pd.pd_workspace_size(c)
    assert n > 2 * 28 * cfg["capacity"]
    bad = pd.config_from_dict(dict(cfg, nz=1))
    with pytest.raises(pd.PdError):
        pd.pd_workspace_size(bad)
    bad = pd.config_from_dict(dict(cfg, field_on=1))      # Poisson needs r-z
    with pytest.raises(pd.PdError):
        pd.pd_workspace_size(bad)
    c2 = pd.config_from_dict(dict(cfg))
    c2.struct_size = 8
    with pytest.raises(pd.PdError):
        pd.pd_workspace_size(c2)


def test_kernel_names():
    assert [pd.pd_kernel_name(k) for k in range(pd.PD_NKERNELS)] == pd.KERNEL_NAMES
