"""The multi-process (N > 1) paths of bench.py, on CPU: two ranks over gloo.

Under torch.distributed.run every rank steps its own replica (no data-path
collective; the geometry does not shard), the timing is the maximum over ranks
and the value counts every rank's node updates.  These tests run bench.py's own
helpers in two spawned processes with the gloo backend (127.0.0.1), and the
reference arm's rule that ranks other than 0 exit without work.
"""
import argparse
import multiprocessing as mp
import os
import socket
import sys
from pathlib import Path

ROOT = str(Path(__file__).resolve().parents[1])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    try:
        r, w, local = bench.dist_init()
        bench.barrier(w)
        ms = 100.0 + 50.0 * r               # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, w)
        value = bench.throughput(1000, 10, w, ms_max)
        bench.barrier(w)
        q.put((r, w, local, dist.get_backend(), ms_max, value))
        dist.destroy_process_group()
    except Exception as e:  # report instead of hanging the parent
        q.put(("error", rank, repr(e)))


def test_two_ranks_max_time_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[0] != "error" for o in out), out
    out.sort()
    for r, (rank, ws, local, backend, ms_max, value) in enumerate(out):
        assert (rank, ws, local, backend) == (r, 2, r, "gloo")
        assert ms_max == 150.0                        # the slowest rank's time
        assert abs(value - 1000 * 10 * 2 / 0.150) < 1e-6  # all ranks' updates / that time


def test_reference_arm_other_ranks_exit_without_work(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(workload="bumpy_h64", steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, ws=2)   # returns at once, prints nothing
    assert capsys.readouterr().out == ""


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = dict(os.environ)
    try:
        os.environ.pop("WORLD_SIZE", None)
        assert bench.dist_init() == (0, 1, 0)
        assert bench.max_over_ranks(3.0, 1) == 3.0
        assert bench.throughput(10, 2, 1, 1000.0) == 20.0
    finally:
        os.environ.clear()
        os.environ.update(env)
