"""Host logic of the benchmark (no GPU): the byte model behind the per-kernel
GB/s and the roofline, the update count of a run, and the digest that keeps a
measured DRAM-traffic figure attached to the push source it was taken on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CSRC = "paper_2109_00214_gb300/csrc/"


def _tree_reader(edits=None):
    """Reads files of the working tree, with `edits` = {relpath: f(text) -> text}."""
    edits = edits or {}

    def read(rel):
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            text = f.read()
        return edits[rel](text) if rel in edits else text
    return read


def test_push_digest_follows_the_push_source_only():
    base = bench.push_source_digest(_tree_reader())
    assert base is not None and len(base) == 64
    # an edit in the sort kernels (after the push section) leaves the digest
    after_sort = _tree_reader({CSRC + "pd_stream.cu": lambda t: t.replace(
        "__global__ void __launch_bounds__(256) k_ebins(", "// edit\n__global__ void __launch_bounds__(256) k_ebins(", 1)})
    assert bench.push_source_digest(after_sort) == base
    # an edit in the push kernel, its launcher or a header changes it
    in_push = _tree_reader({CSRC + "pd_stream.cu": lambda t: t.replace(
        "k_push4(Particles A", "k_push4(Particles  A", 1)})
    assert bench.push_source_digest(in_push) != base
    in_launcher = _tree_reader({CSRC + "pd_stream.cu": lambda t: t.replace(
        "const bool rz = P.geom == 0, field = P.field_on != 0;",
        "const bool rz = P.geom == 0,  field = P.field_on != 0;", 1)})
    assert bench.push_source_digest(in_launcher) != base
    in_header = _tree_reader({CSRC + "pd_internal.cuh": lambda t: t + "\n"})
    assert bench.push_source_digest(in_header) != base
    # a file without the push section has no digest
    assert bench.push_source_digest(lambda rel: "") is None


def test_traffic_figure_only_for_the_captured_source(monkeypatch):
    monkeypatch.setattr(bench, "push_source_digest", lambda read=None: bench.TRAFFIC_SOURCE_SHA)
    assert bench.traffic_per_particle("push") == pytest.approx(796.619e6 / 24898326)
    assert bench.traffic_per_particle("collide") is None
    monkeypatch.setattr(bench, "push_source_digest", lambda read=None: "0" * 64)
    assert bench.traffic_per_particle("push") is None


def test_update_count_of_a_run():
    # 10 steps, heavies every 5th: electrons 10 times, heavies twice,
    # each at the mean of the populations at the start and the end
    c0 = [100, 50, 20, 0, 0, 0, 0]
    c1 = [120, 48, 22, 0, 0, 0, 0]
    assert bench.step_updates(c0, c1, 10, 5) == pytest.approx(10 * 110 + 2 * 70)
    assert bench.step_updates(c0, c1, 10, 1) == pytest.approx(10 * 110 + 10 * 70)


def test_kernel_byte_model():
    steps, n_e, n_h, slots, cand, ncell = 4, 1000.0, 9000.0, 11000.0, 50.0, 256
    prof = {"push": (2.0, 4), "scatter": (1.0, 36), "collide": (0.5, 12), "finalize": (0.1, 4), "idle": (0.0, 0)}
    t = bench.kernel_table(prof, steps, n_e + n_h, n_e, n_h, 1, slots, cand, ncell, 3 * ncell, False, 6000.0)
    assert "idle" not in t
    # Cartesian push: 56 B per electron, 28 B per heavy particle, 4 B per slack slot
    push_bytes = 56 * n_e + 28 * n_h + 4 * (slots - n_e - n_h)
    assert t["push"]["algorithmic_bytes_per_step"] == pytest.approx(push_bytes)
    assert t["push"]["GBs"] == pytest.approx(push_bytes / (0.5e-3) / 1e9)
    assert t["push"]["frac_of_peak"] == pytest.approx(t["push"]["GBs"] / 6000.0)
    assert t["push"]["launches_per_step"] == 1.0
    # the sort: every electron read and written (56 B), 8 B per heavy bin
    assert t["scatter"]["algorithmic_bytes_per_step"] == pytest.approx(56 * n_e + 8 * 3 * ncell)
    assert t["collide"]["algorithmic_bytes_per_step"] == pytest.approx(100 * cand)
    assert "GBs" not in t["finalize"] and t["finalize"]["ms_per_step"] == pytest.approx(0.025)
    # r-z with the field: a heavy particle 44 B on its heavy step, its key (4 B) on the others
    t = bench.kernel_table(prof, steps, n_e + n_h, n_e, n_h, 10, slots, cand, ncell, 3 * ncell, True, 6000.0)
    rz = 56 * n_e + n_h * (44 + 4 * 9) / 10 + 4 * (slots - n_e - n_h)
    assert t["push"]["algorithmic_bytes_per_step"] == pytest.approx(rz)
