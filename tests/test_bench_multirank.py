"""The bench's multi-rank bookkeeping on CPU: two gloo ranks agree on the
slowest rank's step time and on the whole-job throughput (replicas, weak
scaling).  No GPU is involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    ms = bench.reduce_max(10.0 + 5.0 * rank, torch.device("cpu"))
    rate = bench.whole_job_mops(1_000_000, w, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, ms, rate))


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_agree_on_the_slowest_step(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == list(range(world))
    for r, w, lr, ms, rate in out:
        assert w == world and lr == r
        assert ms == 10.0 + 5.0 * (world - 1)                 # the slowest rank
        assert abs(rate - world * 1.0 / (ms / 1e3)) < 1e-9    # 1e6 units per rank, in M/s


def test_single_process_reduce_is_identity():
    import torch
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu")) == 3.5
    assert bench.whole_job_mops(2_000_000, 1, 2.0) == 1000.0
