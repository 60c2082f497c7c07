"""The allocation-free spectrum entry point (pd_energy_spectrum_static).

It serves callers that keep particles in their own device buffers and cannot
allocate device memory for a diagnostic.  Its histogram scratch is a fixed
array inside the library, shared by all calls.  This test feeds it the raw
arrays of a running simulation and checks it against pd_get_energy_spectrum
(which uses the simulation's workspace) on two calls in a row.  The second
call reuses the scratch the first one filled, so stale counts would show.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def test_static_spectrum_matches_workspace_spectrum():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00214_gb300 as pd

    xs = synthetic.standin_cross_sections()
    cfg, parts = synthetic.microbench(nz=48, nr=40, total=1.2e5, coll_scale=3000.0, seed=21)
    sim = pd.Simulation(cfg, xs)
    sim.load(parts)
    sim.step(2)                                  # spawns, conversions and dead slots
    g = sim.particles(live_only=False)
    key = np.where(g["species"] == 255, np.uint32(0xFFFFFFFF),
                   (g["species"].astype(np.uint32) << 24)
                   | (g["iz"].astype(np.uint32) * np.uint32(cfg["nr"]) + g["ir"].astype(np.uint32)))
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev)
         for k, v in (("key", key.astype(np.uint32).view(np.int32)), ("vz", g["vz"]), ("vr", g["vr"]),
                      ("vt", g["vt"]))}
    n = len(key)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize()

    def static(species, lo, hi, nbins):
        return pd.pd_energy_spectrum_static(t["key"].data_ptr(), t["vz"].data_ptr(), t["vr"].data_ptr(),
                                            t["vt"].data_ptr(), n, species, lo, hi, nbins, stream)

    # call 1: electrons; call 2: neutrals over the same number of bins (any
    # count left over from call 1 would show up here)
    a = static(0, 0.0, 200.0, 400)
    b = static(1, 0.0, 1.0, 400)
    assert a.sum() > 0 and b.sum() > 0
    assert np.array_equal(a, sim.energy_spectrum(0, 0.0, 200.0, 400))
    assert np.array_equal(b, sim.energy_spectrum(1, 0.0, 1.0, 400))
    # sizes beyond the fixed scratch are refused, by the library itself
    big = pd.pd_spectrum_static_max_bins() + 1
    with pytest.raises(pd.PdError):
        static(0, 0.0, 200.0, big)
    out = np.zeros(big, np.uint64)
    r = pd._lib().pd_energy_spectrum_static(pd.P(t["key"].data_ptr()), pd.P(t["vz"].data_ptr()),
                                             pd.P(t["vr"].data_ptr()), pd.P(t["vt"].data_ptr()), n, 0, 0.0, 200.0,
                                             big, pd.P(stream), out.ctypes.data_as(pd.P))
    assert pd.STATUS[r] == "PD_ERR_ARG"
    sim.close()
