"""The benchmark's multi-rank logic on the CPU: world size 2 over gloo (replicas, the
slowest rank's time, the whole-job rate), and the reference arm under torchrun, where
rank 0 alone prints its line."""
import json
import math
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(dist, 10.0 + 3.0 * rank, device="cpu")
    rate = bench.job_rate(ws, 256 ** 3, 10, t)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "rate": rate}, f)


def test_max_over_ranks_and_job_rate_world_size_2(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["t"] == 13.0                       # the slower rank's time, on every rank
        assert math.isclose(r["rate"], 2 * 256 ** 3 * 10 / 13e-3, rel_tol=1e-12)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(None, 4.5) == 4.5
    assert bench.job_rate(1, 100, 2, 1.0) == 2e5


def test_reference_arm_under_torchrun_prints_on_rank_0_only():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
