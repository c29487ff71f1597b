"""The replica path of bench.py on several ranks, on the CPU with gloo (no GPU): the job time is
the slowest rank's, the job rate counts every rank's node updates, and under torchrun the
oracle reference arm runs on rank 0 alone while the other ranks exit cleanly."""
import json
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


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = [12.5, 20.0][rank]
        ms_max = bench.max_over_ranks(local_ms, ws, device="cpu")
        q.put((rank, ms_max, bench.job_mlups(ws, 1000, 10, ms_max)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [20.0, 20.0]
    # 2 ranks x 1000 nodes x 10 steps in 20 ms
    assert got[0][2] == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_prints_the_config_of_the_bench_line():
    """Both arms describe the same workload: the reference line's config is the one the GPU arm
    builds for the same flags (the GPU arm itself needs a GPU; its config comes from the same
    builder)."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
           "--precision", "fp16"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(workload="impact", precision="fp16")
    assert d["config"] == json.loads(json.dumps(
        bench.line_config(args, bench.workload("impact"), 1)))
    assert d["config"]["storage"] == bench.STORAGE["fp16"]
    assert d["metric"] == bench.METRIC and d["unit"] == "MLUPS" and d["higher_is_better"]
