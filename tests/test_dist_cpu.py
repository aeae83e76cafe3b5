"""Multi-rank host logic on CPU with gloo (world size 2): each rank gets its
own noise key, the timing reduction is the maximum over ranks, and the
aggregate rate counts every rank's work over the slowest rank's time."""
import socket

import pytest
import torch.multiprocessing as mp

from paper_0903_3852_gb300 import dist as sde_dist
from paper_0903_3852_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    seed = sde_dist.rank_seed(inputs.josephson_sweep.__defaults__[3], rank)
    ms = 100.0 + 10.0 * rank
    mx = sde_dist.max_over_ranks(ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, seed, mx))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0), (r1, s1, m1) = out
    assert (r0, r1) == (0, 1)
    assert s0 != s1 and s1 - s0 == sde_dist.RANK_SEED_STRIDE
    assert m0 == m1 == 110.0
    assert sde_dist.aggregate_rate(4.0e10, 2, 0.110) == pytest.approx(4.0e10 * 2 / 0.110)


def test_single_process_defaults():
    assert sde_dist.max_over_ranks(3.5) == 3.5
    assert sde_dist.rank_seed(7, 0) == 7
