"""The multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path does not shard inside a scene: N GPUs run N independent replicas,
with a barrier around the timed region, the slowest rank's time (max over
ranks) and the summed Newton iterations of all ranks.  These tests run that
host logic as two CPU processes over gloo, and the reference arm under
torchrun, where rank 0 alone times the oracle and prints the line and the
other rank exits 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, _ = bench.dist_setup(world)
    backend = dist.get_backend()
    bench.barrier(w)
    t_max = bench.allreduce_max(w, 1.5 + r)      # per-rank times 1.5 and 2.5
    n_sum = bench.allreduce_sum(w, 10.0 * (r + 1))  # per-rank iteration counts 10 and 20
    bench.barrier(w)
    dist.destroy_process_group()
    out.put((r, w, backend, t_max, n_sum))


def test_replica_reductions_over_gloo():
    if torch.cuda.is_available():  # with a device the ranks would take NCCL on one GPU
        pytest.skip("CPU-only test (gloo ranks)")
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_replica, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    res = sorted(q.get(timeout=60) for _ in range(2))
    for r, w, backend, t_max, n_sum in res:
        assert w == 2 and backend == "gloo"
        assert t_max == 2.5   # the slowest rank's time
        assert n_sum == 30.0  # work of all ranks
    assert [r for r, *_ in res] == [0, 1]


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
