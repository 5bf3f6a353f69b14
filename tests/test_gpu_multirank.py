"""The multi-GPU split on one GPU: two processes (gloo ranks, both on cuda:0;
their kernels never wait on each other) each walk their share and the
results are combined on rank 0.
  * One permanent: each rank computes perm_c128_range partials of its code
    ranges (App. A distribute, dealt round-robin); the partials, gathered and
    added in fixed rank order, equal perm_c128 of the whole matrix.
  * A batch: multirank.shard_batch deals the matrices by cost; each rank runs
    perm_batch on its shard; the gathered results equal the single-process
    batch bit for bit (each matrix's items and their order depend only on the
    matrix and its order's choices)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

N_RANGE = 27
SEED = 606


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _batch_input():
    from paper_1904_06229_gb300 import workloads as W

    return W.batch_study(80, seed=31, n_lo=10, n_hi=22)


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1904_06229_gb300 import multirank as M
    from paper_1904_06229_gb300 import perm as P
    from paper_1904_06229_gb300 import workloads as W

    A = torch.from_numpy(W.haar_submatrix(N_RANGE, N_RANGE * N_RANGE, SEED)).cuda()
    mine = [P.perm_c128_range(A, f, c).cpu().tolist() for f, c in M.rank_ranges(N_RANGE, world, rank, 3)]
    ns, mats = _batch_input()
    shard = M.shard_batch(ns, world)[rank]
    dm = [torch.from_numpy(np.ascontiguousarray(mats[k])).cuda() for k in shard]
    res = P.perm_batch(dm).cpu().numpy().tolist() if dm else []
    assert P.perm_last_status() == 0
    gathered = [None] * world
    dist.all_gather_object(gathered, {"partials": mine, "shard": shard, "batch": res})
    if rank == 0:
        per = M.combine_partials([g["partials"] for g in gathered], N_RANGE)
        out = [None] * len(ns)
        for g in gathered:
            for k, v in zip(g["shard"], g["batch"]):
                out[k] = v
        q.put({"per": per, "batch": out})
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_one_gpu():
    from paper_1904_06229_gb300 import perm as P
    from paper_1904_06229_gb300 import workloads as W

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    A = torch.from_numpy(W.haar_submatrix(N_RANGE, N_RANGE * N_RANGE, SEED)).cuda()
    ref = P.perm_c128(A).cpu().numpy()
    ref = complex(ref[0], ref[1])
    rel = abs(got["per"] - ref) / abs(ref)
    print(f"two ranks, n={N_RANGE}: combined partials vs perm_c128 rel diff {rel:.3e}")
    assert rel <= 1e-12
    ns, mats = _batch_input()
    whole = P.perm_batch([torch.from_numpy(np.ascontiguousarray(m)).cuda() for m in mats]).cpu().numpy()
    assert np.array_equal(np.asarray(got["batch"]), whole)
