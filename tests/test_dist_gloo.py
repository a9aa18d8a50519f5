"""Multi-process host logic on the CPU (gloo, world size 2): the timing
reduction and whole-job rate of a replicated run, and the round-robin batch
sharding -- the N > 1 path of the benchmark without GPUs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2310_13421_gb300 import dist as tdist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = tdist.rank_env()
        # each rank "timed" a different step time; the job takes the slowest
        my_ms = 10.0 + 5.0 * rank
        slowest = tdist.max_over_ranks(my_ms)
        units = tdist.sum_over_ranks(1000)
        rate = tdist.job_rate(w * 1000, slowest)
        mine = tdist.shard(list(range(11)), r, w)
        seen = [None] * w
        dist.all_gather_object(seen, mine)
        out.put((rank, w, r, lr, slowest, units, rate, sorted(x for part in seen for x in part)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, lr, slowest, units, rate, union in results:
        assert (w, r, lr) == (world, rank, rank)
        assert slowest == 15.0                      # max over ranks
        assert units == 2000.0
        assert rate == pytest.approx(2000 / 15e-3)  # whole-job units / slowest time
        assert union == list(range(11))             # the shards cover the batch once


def test_single_process_fallbacks():
    from paper_2310_13421_gb300 import dist as tdist
    assert tdist.max_over_ranks(3.5) == 3.5
    assert tdist.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    with pytest.raises(ValueError):
        tdist.shard([1], 2, 2)
    with pytest.raises(ValueError):
        tdist.job_rate(1, 0)
