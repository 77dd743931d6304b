"""The multi-rank path of bench.py on CPU (gloo, two ranks): one independent replica
per rank, no collective on the data path, the timed region the slowest rank's, and
the reference arm run by rank 0 alone."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    slowest = bench.max_over_ranks(1.5 * (rank + 1), dist)
    w = bench.load_workload("plain", rank)
    out.put((rank, slowest, int(w["seed"]), tuple(w["grid"]), len(w["q"]), [float(x) for x in w["q"][0]]))
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_take_the_slowest_time_and_their_own_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, rest) for r, *rest in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (s0, seed0, grid0, nb0, q0), (s1, seed1, grid1, nb1, q1) = got[0], got[1]
    assert s0 == s1 == 3.0                           # max over ranks, seen by both
    assert grid0 == grid1 and nb0 == nb1             # the same workload shape on every rank
    assert seed0 != seed1 and q0 != q1               # but an independent replica


def test_reference_arm_runs_on_rank_zero_only():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--workload", "plain", "--steps", "1", "--warmup", "0", "--cpu-budget", "5", "--gpus", "2"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
