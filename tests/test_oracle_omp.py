"""The oracle's OpenMP build (all host cores) against its serial build (no
GPU): the same particles (by id), counters and fixed-point charge, bit for
bit, and the FP64 ledgers to rounding (they are summed in another order).
The OpenMP build collides cells in parallel with each spawn in the slot its
id reserves, pushes particles independently and compacts in order, so a
step is deterministic on any number of threads."""
import numpy as np
import pytest

import oracle
import synthetic


def run(cfg, parts, xs, steps, omp, fp64=False, field=None):
    o = oracle.Oracle(cfg, fp64=fp64, omp=omp)
    o.set_cross_sections(xs)
    if len(parts["species"]):
        o.load(parts)
    if field is not None:
        o.set_field(*field)
    o.prime()
    o.step(steps)
    return o


def same(a, b):
    pa, pb = a.particles(), b.particles()
    oa, ob = np.argsort(pa["id"], kind="stable"), np.argsort(pb["id"], kind="stable")
    assert len(oa) == len(ob)
    for k in pa:
        assert np.array_equal(pa[k][oa], pb[k][ob]), k
    assert a.counters() == b.counters()
    ra, rb = a.rho(), b.rho()
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
    sa, sb = a.scalars(), b.scalars()
    for k in sa:
        assert sa[k] == pytest.approx(sb[k], rel=1e-12, abs=1e-300), k


@pytest.mark.parametrize("fp64", [False, True])
def test_omp_microbench_with_collisions(fp64):
    cfg, parts = synthetic.microbench(nz=24, nr=20, total=3e4, coll_scale=3000.0, seed=5)
    xs = synthetic.standin_cross_sections()
    same(run(cfg, parts, xs, 4, True, fp64), run(cfg, parts, xs, 4, False, fp64))


def test_omp_rz_field_injection_and_extensions():
    cfg, parts = synthetic.rz_plume(n=32, total=2e4, seed=8)
    cfg.update(field_on=1, inject_on=1, beta=1.0, heavy_coll=1, coulomb=1, charge_max=4, heavy_subcycle=2,
               coll_dt_scale=50.0, capacity=1 << 17)
    xs = synthetic.standin_cross_sections()
    same(run(cfg, parts, xs, 6, True), run(cfg, parts, xs, 6, False))


def test_omp_sputtering_keeps_the_serial_push():
    cfg, parts = synthetic.rz_plume(n=32, total=2e4, seed=9)
    cfg.update(field_on=1, inject_on=0, sputter=1, heavy_subcycle=1, capacity=1 << 17)
    xs = synthetic.standin_cross_sections()
    a = oracle.Oracle(cfg, fp64=False, omp=True)
    b = oracle.Oracle(cfg, fp64=False)
    E, Y = synthetic.standin_sputter_yield()
    for o in (a, b):
        o.set_cross_sections(xs)
        o.set_sputter_yield(E, Y)
        o.load(parts)
        o.prime()
        o.step(4)
    same(a, b)
