"""The N>1 host path of bench.py on CPU: two gloo ranks (127.0.0.1) run the same
aggregation the GPU replicas use -- barrier, max of the per-rank timed region, and
the whole-job value (units of all ranks / max time) -- and rank 0 reports it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    d = bench.dist_init(w, use_cuda=False)
    d.barrier()
    ms = 10.0 * (rank + 1)                    # rank-dependent timed region
    ms_max = bench.reduce_max(d, ms)
    total = bench.reduce_sum(d, 1000.0 * (rank + 1))
    value = w * 262144 * 4 * 5 / (ms_max * 1e-3)
    out[rank] = (ms_max, total, value)
    d.barrier()
    d.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0          # max over ranks
    assert out[0][1] == out[1][1] == 3000.0
    assert out[0][2] == pytest.approx(2 * 262144 * 4 * 5 / 0.02)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.dist_init(1, use_cuda=False) is None
    assert bench.reduce_max(None, 3.5) == 3.5
