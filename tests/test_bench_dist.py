"""Replica aggregation of bench.py across ranks, on CPU with torch.distributed gloo (world size 2):
the job's value is the units of all ranks over the slowest rank's time; and the reference arm under
torchrun, where rank 0 alone runs and prints."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 250.0][rank]
    units = [1000.0, 3000.0][rank]
    agg = bench.aggregate(ms, units, steps=10)
    bench.barrier()
    assert bench.dist_env() == (rank, rank, world)
    out.put((rank, agg))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r]["ms"] == 250.0
        assert res[r]["units"] == 4000.0
        assert abs(res[r]["value"] - 4000.0 * 10 / 0.25) < 1e-6


def test_single_process_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    agg = bench.aggregate(50.0, 200.0, steps=4)
    assert agg["ms"] == 50.0 and agg["value"] == 200.0 * 4 / 0.05


def test_reference_arm_under_torchrun_two_ranks():
    # bench.py --impl reference launched as the multi-GPU command is: rank 0 alone times the oracle
    # (here on 2 host threads, one slab each) and prints one JSON line; rank 1 exits 0 with no output
    import json
    import subprocess
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-threads", "2"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
