"""bench.py's multi-rank path on CPU (gloo, world size 2): replicas time
their own work, the slowest rank's time is shared, and the whole-job
throughput counts every rank's work; the reference arm prints on rank 0
only."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 2.0 + rank  # rank 1 is the slow one
    m = bench._max_over_ranks(ms, ws, device="cpu")
    bench._barrier(ws)
    q.put((rank, m, bench.whole_job_rate(1e12, m, ws)))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.0, 3.0]
    assert res[0][2] == pytest.approx(2 * 1e12 / 3e-3)


def _ref_worker(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import bench
    printed = []

    class A:
        gpus, steps, warmup = ws, 1, 0

    import builtins
    orig = builtins.print
    builtins.print = lambda *a, **k: printed.append(a)
    try:
        if rank != 0:
            bench.run_reference(A, rank, ws)  # returns without work
    finally:
        builtins.print = orig
    q.put((rank, len(printed)))


def test_reference_arm_nonzero_ranks_do_nothing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_ref_worker, args=(1, 2, _free_port(), q))
    p.start()
    rank, n = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0 and n == 0


def test_recorded_traffic_only_for_its_size_and_sources(tmp_path):
    """The roofline's DRAM traffic comes from the committed ncu record only for
    the product size it was captured on and while the kernel's sources hash
    to the recorded value; anything else reports null."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    rec = {"tc_gemm_pair<3>": {"n": 8192, "source_sha256": bench.kernel_source_hash(), "dram_bytes_per_launch": 123}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    assert bench._ncu_traffic("tc_gemm_pair<3>", 8192, path=str(p)) == 123
    assert bench._ncu_traffic("tc_gemm_pair<3>", 1024, path=str(p)) is None
    assert bench._ncu_traffic("tc_gemm_pair<0>", 8192, path=str(p)) is None
    rec["tc_gemm_pair<3>"]["source_sha256"] = "0" * 64
    p.write_text(json.dumps(rec))
    assert bench._ncu_traffic("tc_gemm_pair<3>", 8192, path=str(p)) is None
