"""Sharding a batch of independent systems across ranks (CPU, gloo).

Two ranks (spawned processes, gloo on 127.0.0.1) each solve their share of
a small batch of 2-D IgA systems, assigned by stored entries, and gather
the results; the union must equal the single-process solve of every system
bit for bit (each system is solved by the same deterministic solver,
wherever it runs).  The per-rank solver here is the CPU oracle, standing in
for the GPU batch hierarchy, which cannot run without a GPU; what is tested
is the sharding and the gather.
"""
import os
import socket

import numpy as np
import pytest

from paper_2511_21268_gb300 import dist as D
from paper_2511_21268_gb300 import inputs as I


def test_assignment_balances_nnz_and_covers_every_system():
    nnz = [50, 10, 40, 40, 5, 30, 20]
    parts = D.assign_by_nnz(nnz, 3)
    assert sorted(k for p in parts for k in p) == list(range(len(nnz)))
    loads = [sum(nnz[k] for k in p) for p in parts]
    assert max(loads) - min(loads) <= max(nnz)
    assert parts == D.assign_by_nnz(nnz, 3)  # deterministic
    assert D.assign_by_nnz(nnz, 1) == [list(range(len(nnz)))]
    assert D.assign_by_nnz([7, 7], 4) == [[0], [1], [], []]


def _batch():
    out = []
    for k, (d, n, p) in enumerate([(2, 8, 2), (2, 12, 3), (2, 10, 2), (2, 6, 4), (2, 14, 2)]):
        q = I.poisson_box_random_rhs(d, n, p, seed=30 + k)
        out.append(q)
    return out


def _oracle_solve(systems, rhs):
    import oracle as O

    res = []
    for (rp, ci, v), F in zip(systems, rhs):
        r = O.Hierarchy(rp, ci, v, coarse_max=20).pcg(F, rtol=1e-10)
        res.append({"u": r["u"], "iters": r["iters"], "status": r["status"]})
    return res


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        probs = _batch()
        systems = [(p.rowptr, p.col, p.val) for p in probs]
        out = D.solve_sharded(systems, [p.F for p in probs], _oracle_solve, rank, world, dist)
        if rank == 0:
            q.put([(o["u"], o["iters"], o["status"]) for o in out])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_the_single_process_batch():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    probs = _batch()
    ref = _oracle_solve([(p.rowptr, p.col, p.val) for p in probs], [p.F for p in probs])
    assert len(got) == len(ref)
    for (u, it, st), r in zip(got, ref):
        assert st == 0 and it == r["iters"]
        assert np.array_equal(u.view(np.uint64), r["u"].view(np.uint64))
