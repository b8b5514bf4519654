"""The multi-GPU path of bench.py is replicas only (independent copies of the
workload, one per rank, no data-path collective): its job time is the
slowest rank's time and its rate counts every rank's cell-steps.  Checked
here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench

    r, w, lr = bench.dist_info()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    ms, value = bench.aggregate(10.0 * (r + 1), cells=1000, steps=4, world=w)
    q.put((r, ms, value))
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_cells():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ms, value in out:
        assert ms == pytest.approx(20.0)  # the slower rank
        assert value == pytest.approx(2 * 1000 * 4 / 0.020 / 1e6)


def test_single_process_aggregate_is_local():
    import bench

    ms, value = bench.aggregate(5.0, cells=100, steps=10, world=1)
    assert ms == 5.0 and value == pytest.approx(100 * 10 / 0.005 / 1e6)
