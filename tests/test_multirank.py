"""The multi-GPU form is independent replicas (no collective on the data path);
what the benchmark does across ranks -- barrier, max of the timed region over
ranks, whole-job throughput, rank 0 alone printing -- is checked here with
world_size-2 gloo process groups on CPU."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    got = bench.max_over_ranks(local_ms, world)
    q.put((rank, got, bench.job_msamples_per_s(1_000_000, 4, world, got)))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    res = sorted(q.get(timeout=60) for _ in range(2))
    assert [r[0] for r in res] == [0, 1]
    # every rank sees the slowest rank's time
    assert all(r[1] == 15.0 for r in res)
    # whole-job value: both ranks' samples over the slowest rank's time
    assert res[0][2] == pytest.approx(2 * 4 * 1_000_000 / 0.015 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_msamples_per_s(8_125_000, 2, 1, 1000.0) == pytest.approx(16.25)


def test_reference_arm_under_torchrun_prints_once():
    """--impl reference with two ranks: rank 0 alone times the oracle and
    prints one JSON line; rank 1 exits 0 without work."""
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1",
           "--cells", "256:4", "--seconds", "0.002", "--ref-seconds", "1"]
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
