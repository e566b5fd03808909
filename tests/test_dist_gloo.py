"""The N > 1 path of bench.py on CPU: two ranks under the gloo backend (a
process each, rendezvous on 127.0.0.1).  Each rank decodes lists of its own
(distinct seeds, no data exchanged); the reported time is the maximum over
the ranks and the rate counts every rank's integers."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    import bench
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world)
        # the slowest rank's time is the job's time
        ms = bench.max_over_ranks(dist, 1.0 + rank)
        bench.barrier(dist)
        # each rank's lists come from its own seeds
        lists = bench.make_lists("uniform", 2, 4096, 1 << 20, bench.rank_seed(rank))
        sums = [int(x.astype(np.uint64).sum()) for x in lists]
        gathered = [None] * world
        dist.all_gather_object(gathered, (rank, bench.rank_seed(rank), sums))
        rate = bench.whole_job_rate(world, 1 << 20, ms)
        q.put((rank, ms, gathered, rate))
        dist.destroy_process_group()
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), None))


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, gathered, rate in out:
        assert ms != "error", gathered
        assert ms == 2.0                       # max over ranks 1.0 and 2.0
        assert rate == pytest.approx(2 * (1 << 20) / 2.0e-3 / 1e9)
        seeds = [g[1] for g in gathered]
        assert len(set(seeds)) == world        # distinct per-rank workloads
        assert gathered[0][2] != gathered[1][2]
    assert out[0][2] == out[1][2]              # both ranks saw the same exchange
