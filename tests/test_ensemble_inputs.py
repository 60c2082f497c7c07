"""The batched-ensemble input recipe: 64 runs (8 seeds x 8 gap voltages),
grids and particle counts drawn per run, accepted by the library as one
ensemble (the size query needs no GPU)."""
import numpy as np

import synthetic


def test_ensemble_recipe_shape_and_determinism():
    runs = synthetic.ensemble_breakdown(seeds=range(1, 9))
    assert len(runs) == 64
    again = synthetic.ensemble_breakdown(seeds=[1])
    for (c, p), (c2, p2) in zip(runs[:8], again):
        assert c == c2
        assert all(np.array_equal(p[k], p2[k]) for k in p)
    grids = [c["nz"] for c, _ in runs]
    assert set(grids) <= set(synthetic.ENSEMBLE_GRIDS) and len(set(grids)) >= 4
    counts = np.array([len(p["species"]) for _, p in runs])
    assert counts.min() >= 0.8e5 and counts.max() <= 2.2e6
    assert len({(c["seed"], c["V0"]) for c, _ in runs}) == 64
    assert sorted({c["V0"] for c, _ in runs}) == [v * 1e3 for v in synthetic.ENSEMBLE_VOLTS_KV]
    for c, p in runs:
        assert c["nz"] == c["nr"] and c["field_on"] == 1 and c["inject_on"] == 0
        assert p["iz"].max() < c["nz"] and p["ir"].max() < c["nr"]
        assert c["capacity"] >= len(p["species"])


def test_library_accepts_the_ensemble():
    import paper_2109_00214_gb300 as pd
    pd.load_library()
    cfgs = [c for c, _ in synthetic.ensemble_breakdown(seeds=range(1, 9), n_lo=10, n_hi=20)]
    n = pd.pd_ensemble_workspace_size([pd.config_from_dict(c) for c in cfgs])
    assert n > 0
