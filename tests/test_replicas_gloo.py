"""The multi-GPU path of the bench is replicas only (independent runs per
rank, no data-path collective): its rank arithmetic -- the split of an
ensemble's runs over ranks, the max-over-ranks time and the summed updates --
checked with two gloo ranks on the CPU, and the reference arm launched by
torchrun with two ranks (rank 0 prints the one JSON line, rank 1 exits 0)."""
import json
import multiprocessing as mp
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo")
    import bench
    m = bench.max_over_ranks(ws, 10.0 * (rank + 1))
    t = bench.sum_over_ranks(ws, float(rank + 1))
    part = bench.shard(list(range(11)), rank, ws)
    bench.barrier(ws)
    q.put((rank, m, t, part))
    dist.destroy_process_group()


def test_rank_arithmetic_with_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]            # max over ranks
    assert [o[2] for o in out] == [3.0, 3.0]              # sum over ranks
    parts = [o[3] for o in out]
    assert sorted(parts[0] + parts[1]) == list(range(11)) and not set(parts[0]) & set(parts[1])


def test_reference_arm_under_torchrun_two_ranks():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--nz", "256", "--nr", "64", "--total", "6e4",
           "--cpu-rows", "16", "--cpu-steps", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
