"""Replica launch path of bench.py on the CPU (gloo, two ranks).

Every GPU of a multi-GPU run solves its own system (replicas, no collective on
the data path); the job's time per step is the slowest rank's.  Two spawned
processes check the process-group set-up that torchrun's environment drives,
the max-over-ranks reduction, and that the reference arm runs on rank 0 only.
"""

import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, local = bench.dist_setup()
    slow = bench.max_over_ranks(10.0 + 5.0 * r, w)
    q.put((r, w, local, dist.get_backend(), slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for r, w, local, backend, slow in got:
        assert w == 2 and local == r and backend == "gloo"
        assert slow == 15.0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    args = bench.parse()
    bench.reference_arm(args, 2, 1)        # rank 1 of 2: no work, no output
    assert capsys.readouterr().out == ""
