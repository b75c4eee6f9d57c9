"""The N > 1 path of bench.py (replicas: one independent system per rank,
no data exchanged) on CPU processes with the gloo backend, world size 2:
the barrier, the max-over-ranks time, the per-rank seeds and the reference
arm's rank-0-only output under torchrun."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w, lr = bench.dist_setup("gloo")
    bench.barrier(w)
    got = bench.max_over_ranks(10.0 * (r + 1), w)
    seeds = [bench.replica_seed(2, k) for k in range(w)]
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((r, w, lr, got, seeds))


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_barrier_and_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    # every rank reports the slowest rank's time
    assert all(o[3] == 20.0 for o in out)
    # each rank solves its own system
    assert out[0][4] == out[1][4] and len(set(out[0][4])) == 2


def test_reference_arm_prints_on_rank0_only():
    """torchrun with 2 CPU processes: rank 0 times the oracle on a small
    sample and prints one JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-seconds", "0.5", "--workload",
           "hpl_f64_n1024_nb64"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    import json
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
