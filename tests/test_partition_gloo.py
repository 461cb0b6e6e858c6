"""The paper's row-partitioned all-at-once loop on CPU ranks (gloo, world size 2).

Each rank computes the outer-product contributions of its block of fine rows
(the oracle's row-block product), sends the rows of C it does not own to their
owners (C_s of Alg. 7-8) and adds what it receives; the assembled rows must
equal the full product.  The remote rows of P each rank needs (P~_r) are
checked against the paper's worked example (Section 2, Eq. 5).
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1905_08423_gb300 import partition as pt
from paper_1905_08423_gb300 import problems as pb


def test_block_bounds_and_owner():
    b = pt.block_bounds(10, 3)
    np.testing.assert_array_equal(b, [0, 4, 7, 10])
    np.testing.assert_array_equal(pt.owner_of([0, 3, 4, 6, 7, 9], b), [0, 0, 1, 1, 2, 2])
    assert pt.block_bounds(2, 4).tolist() == [0, 1, 2, 2, 2]


def test_remote_rows_eq5():
    """Section 2, Eq. 5: the first of three processes (rows 1-2) needs remote rows 3 and 5."""
    rows = [[0, 1, 4], [1, 2, 4], [0, 3, 4], [1, 3], [3, 4], [1, 4, 5]]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    A = pb.CSR(6, 6, rp, np.concatenate(rows).astype(np.int32), np.ones(rp[-1]))
    np.testing.assert_array_equal(pt.remote_rows(A, 0, 2), [2, 4])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, P = pb.algebraic_problem(9, seed=6)
        fb = pt.block_bounds(A.nrows, world)
        cb = pt.block_bounds(P.ncols, world)
        r0, r1 = int(fb[rank]), int(fb[rank + 1])
        local = oracle.ptap_row_block(A, P, r0, r1)     # contributions of my fine rows
        nz = np.nonzero(np.diff(local.row_ptr))[0]
        sub_rp = np.concatenate([[0], np.cumsum(np.diff(local.row_ptr)[nz])])
        idx = np.concatenate([np.arange(local.row_ptr[i], local.row_ptr[i + 1]) for i in nz]) if len(nz) else []
        msgs = pt.split_by_owner(nz, sub_rp, local.col_idx[idx], local.val[idx], cb)
        gathered = [None] * world
        dist.all_gather_object(gathered, msgs)
        mine = [g[rank] for g in gathered if rank in g]
        c0, c1 = int(cb[rank]), int(cb[rank + 1])
        rp, ci, v = pt.assemble(mine, c0, c1)
        full = oracle.ptap(A, P)
        ok = (np.array_equal(rp, full.row_ptr[c0:c1 + 1] - full.row_ptr[c0])
              and np.array_equal(ci, full.col_idx[full.row_ptr[c0]:full.row_ptr[c1]])
              and np.allclose(v, full.val[full.row_ptr[c0]:full.row_ptr[c1]], rtol=1e-12, atol=1e-12))
        q.put((rank, bool(ok), len(pt.remote_rows(A, r0, r1))))
    finally:
        dist.destroy_process_group()


def test_two_rank_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert sorted(r[0] for r in res) == [0, 1]
    assert all(r[1] for r in res), res
    assert all(r[2] > 0 for r in res)   # each half needs rows of P from the other
