"""Multi-process (replica) host logic of bench.py on CPU with gloo, world size 2.

The evaluation has no exchange step, so N GPUs run N independent replicas;
the only collectives are the barriers around the timed region and the
max-over-ranks reduction of the step time.  These tests run that logic in two
gloo processes, and the reference arm under torchrun (rank 0 prints one
line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"WORLD_SIZE": str(world), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.init_replicas("gloo")
    assert bench.ranks() == (world, rank, rank)
    dist.barrier()
    slowest = bench.max_over_ranks(1.5 + rank, dist)  # rank r "took" 1.5 + r ms
    value = bench.replica_throughput(world, 1000, slowest / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, slowest, value))


def test_max_over_ranks_and_weak_throughput_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in res:
        assert slowest == 2.5                       # the slower rank's time on both
        assert value == pytest.approx(2 * 1000 * 1000 / 2.5e-3)  # 2 replicas x N^2


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.init_replicas("gloo") is None
        assert bench.max_over_ranks(3.25, None) == 3.25
        assert bench.replica_throughput(1, 10, 2.0) == 50.0
    finally:
        os.environ.update(env)


def test_reference_arm_under_torchrun_world2():
    """bench.py --impl reference launched like the multi-GPU driver run: one
    JSON line from rank 0 with the reference keys, exit 0 on both ranks."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--points", "2000",
           "--cpu-targets", "4"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300,
                       env={**os.environ, "OMP_NUM_THREADS": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
