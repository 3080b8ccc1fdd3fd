"""The multi-rank path of bench.py on CPU (gloo, world size 2).

The apply shards by right-hand sides with no exchange: each rank runs its own
replica and batch, and the job's throughput is every rank's units over the
slowest rank's time.  Here two gloo ranks check that reduction and the
aggregate on the host, and that the oracle's reference arm does no work on
ranks other than 0."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, w)     # rank 1 is the slow one
    rate = bench.aggregate_rate(64 * 20, w, slowest)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, slowest, rate))


def test_max_over_ranks_and_the_aggregate_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == 15.0 for o in out)                    # every rank sees the slowest time
    assert all(o[4] == pytest.approx(2 * 64 * 20 / 15.0) for o in out)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(100, 1, 2.0) == 50.0


def test_reference_arm_is_idle_off_rank_0():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "fp32_512"
        steps = 1
        warmup = 1
        gpus = 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args(), 1, 2) is None
    assert buf.getvalue() == ""
