"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its own
independent solve (replicas; the solve itself has no collective), must agree
on the slowest rank's time, which is what the JSON line reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, results):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench._dist_env()
        assert (w, r, loc) == (world, rank, rank)
        bench._barrier(True)
        ms = 10.0 + 5.0 * rank                  # rank 1 is the slow one
        results[rank] = bench._max_over_ranks(ms, True, torch.device("cpu"))
        bench._barrier(True)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        assert dict(results) == {0: 15.0, 1: 15.0}


def test_single_process_defaults():
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench._dist_env() == (1, 0, 0)
    assert bench._max_over_ranks(3.5, False, None) == 3.5
