"""The N > 1 path on CPU: two ranks over gloo (127.0.0.1).

Replicas only: every rank solves its own systems (its own seed) with no
data-path collective; the job's time is the slowest rank's (max over ranks,
all ranks agree), and the whole-job rate counts the units of all ranks.
With the environment torchrun sets, the reference arm runs on rank 0 alone
and the other ranks exit 0 without output.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="env://")
    try:
        import bench
        import workloads as W
        w, r, local = bench.dist_env()
        slowest = bench.reduce_max(10.0 + 5.0 * r, w, "cpu")       # this rank's "time"
        rate = bench.job_rate(w, 3, slowest)
        A, _, _ = W.svd_kappa(64, 1e2, 1, seed=0 + r)               # the replica's own system
        digests = [None] * w
        dist.all_gather_object(digests, float(A.double().sum()))
        dist.barrier()
        q.put((r, w, local, slowest, rate, digests))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, w, local, slowest, rate, digests) in enumerate(out):
        assert (rank, w, local) == (r, 2, r)
        assert slowest == 15.0                       # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 3 / 0.015)  # units of both ranks over that time
        assert digests[0] != digests[1]              # each replica solves its own system
    assert out[0][5] == out[1][5]


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(1, 8, 4000.0) == 2.0


def test_reference_arm_two_ranks_prints_once():
    """Two ranks with the environment torchrun gives them (RANK, WORLD_SIZE,
    LOCAL_RANK, MASTER_*): rank 0 times the oracle and prints the one line,
    rank 1 exits 0 without output."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        cmd = [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--workload", "lead", "--n", "128",
               "--nrhs", "1", "--steps", "1", "--warmup", "0"]
        procs.append(subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    assert [p.returncode for p in procs] == [0, 0], [o[1][-2000:] for o in outs]
    lines0 = [l for l in outs[0][0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1][0].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    line = json.loads(lines0[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
