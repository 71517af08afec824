"""The multi-process path of bench.py on CPU (gloo, world size 2): process
group set-up from the launcher's environment, the barrier, the max over
ranks of the step time, and the whole-job rate (units of every rank over the
slowest rank's time).  The GPU path is the same code with NCCL."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, root, out):
    sys.path.insert(0, root)
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, w)
    out[rank] = (ms_max, bench.job_throughput(9, ms_max, w))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, ROOT, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for r in range(2):
        ms_max, rate = out[r]
        assert ms_max == 15.0
        assert rate == pytest.approx(2 * 9 / 15e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(9, 40.0, 1) == pytest.approx(225.0)
