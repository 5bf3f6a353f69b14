"""Multi-rank path on CPU: two gloo ranks split one permanent's Gray range,
gather their partials and combine them in fixed rank order.  The per-range
partials come from the oracle here (no GPU in this process); on GPUs each rank
calls perm_c128_range instead."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_06229_gb300 import multirank as M


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, seed, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_1904_06229_gb300 import workloads as W

    A = W.complex_gaussian(n, seed)
    mine = []
    for first, count in M.rank_ranges(n, world, rank, pieces_per_rank=3):
        g = O.glynn_partial(A, first, count)
        re, im = float(g[0]), float(g[1])
        mine.append([re, float(g[0] - np.longdouble(re)), im, float(g[1] - np.longdouble(im))])
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        q.put(M.combine_partials(gathered, n))
    dist.barrier()
    dist.destroy_process_group()


def test_distribute_covers_range():
    for total, parts in ((1 << 19, 7), (10, 3), (5, 8)):
        pieces = [M.distribute(total, parts, i) for i in range(parts)]
        assert pieces[0][0] == 0
        for (a, b), (c, _) in zip(pieces[:-1], pieces[1:]):
            assert a + b == c
        assert sum(b for _, b in pieces) == total
    rr = [M.rank_ranges(9, 2, r, 3) for r in range(2)]
    allr = sorted(x for r in rr for x in r)
    assert allr[0][0] == 0 and sum(c for _, c in allr) == 1 << 8


def test_two_gloo_ranks_combine_to_permanent():
    from oracle import oracle as O
    from paper_1904_06229_gb300 import workloads as W

    n, seed, world = 13, 21, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    r = O.per(W.complex_gaussian(n, seed))
    ref = complex(float(r[0]), float(r[1]))
    assert abs(got - ref) <= 1e-14 * abs(ref)


def test_dd_add_exact_cancellation():
    a = (1.0, 1e-20)
    b = (-1.0, 3e-20)
    s = M.dd_add(a, b)
    assert s[0] + s[1] == pytest.approx(4e-20, rel=1e-12)


def test_shard_batch_balances_cost():
    from paper_1904_06229_gb300 import workloads as W

    ns = W.batch_sizes(5000, 3)
    for world in (1, 2, 3, 8):
        shards = M.shard_batch(ns, world)
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(len(ns)))  # every matrix exactly once
        loads = [sum(1 << (int(ns[k]) - 1) for k in s) for s in shards]
        # greedy deal in decreasing cost: the spread is at most the largest item
        assert max(loads) - min(loads) <= 1 << (int(max(ns)) - 1)
        assert max(loads) <= sum(loads) / world + (1 << (int(max(ns)) - 1))


def test_shard_batch_small_cases():
    assert M.shard_batch([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]
    assert M.shard_batch([5], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        M.shard_batch([4], 0)
