"""The paper's row-partitioned all-at-once product (Section 2, Eq. 1-3; Alg. 7-10)
on CPU ranks.

Each rank holds only its block of fine rows of A and P.  It gathers the rows
of P its block references elsewhere (P~_r) from their owners, runs its local
product, sends the contributions to coarse rows it does not own (C_s) to
their owners and adds what it receives.  The assembled owned rows of C must
equal the oracle's full product -- pattern exactly, values within 1e-12 of
|P|^T|A||P| -- for the merged loop (Alg. 9-10) and the remote-first loop
(Alg. 7-8), on gloo ranks (world size 2 and 3) and in lockstep in one
process (world size 4).  The local products here run on the oracle; the GPU
test of the same driver runs them in the CUDA library.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1905_08423_gb300 import partition as pt
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import sharded as sh


class OracleOps:
    """Test backend: the oracle runs each rank's local product; torch CPU tensors carry values."""

    dtype = torch.float64

    def comm_i64(self, x):
        return torch.as_tensor(np.asarray(x, dtype=np.int64))

    def np(self, t):
        return t.numpy().astype(np.int64)

    def index(self, x):
        return torch.as_tensor(np.asarray(x, dtype=np.int64))

    def plan(self, A_part, P_ext):
        C = oracle.ptap(A_part, P_ext)
        return (A_part, P_ext, C.nnz), C.row_ptr, C.col_idx

    def allocate(self, p):
        p.p_ext_vals = torch.empty(p.p_ext_nnz, dtype=self.dtype)
        for part in p.parts:
            part.c_vals = torch.empty(part.plan[2], dtype=self.dtype)
        p.c_own = torch.empty(int(p.own_rp[-1]), dtype=self.dtype)

    def empty(self, n):
        return torch.empty(n, dtype=self.dtype)

    def gather(self, src, idx):
        return src[idx].clone()

    def scatter_add(self, dst, dst_idx, src, src_idx=None):
        v = src[src_idx] if src_idx is not None else src[:dst_idx.numel()]
        dst.index_add_(0, dst_idx, v)

    def copy(self, dst, src):
        dst.copy_(src)

    def zero(self, t):
        t.zero_()

    def numeric(self, plan, A_vals, P_vals, out):
        A_part, P_ext, _ = plan
        C = oracle.ptap(A_part.with_values(A_vals.numpy()), P_ext.with_values(P_vals.numpy()))
        out.copy_(torch.as_tensor(C.val))


def _problem(kind):
    return pb.algebraic_problem(9, seed=6) if kind == "algebraic" else pb.model_problem(11)


def _check_rows(A, P, c0, c1, own_rp, own_ci, vals):
    full = oracle.ptap(A, P)
    bnd = oracle.ptap_bound(A, P)
    a, b = full.row_ptr[c0], full.row_ptr[c1]
    np.testing.assert_array_equal(own_rp, full.row_ptr[c0:c1 + 1] - a)
    np.testing.assert_array_equal(own_ci, full.col_idx[a:b])
    err = np.abs(np.asarray(vals, dtype=np.float64) - full.val[a:b])
    assert np.all(err <= 1e-12 * bnd.val[a:b] + (bnd.val[a:b] == 0) * 0.0)


def _rank_gens(A, P, world, merged, scale=None):
    """Per rank: setup and numeric generators over that rank's blocks only."""
    fb = pt.block_bounds(A.nrows, world)
    gens, vals = [], []
    for r in range(world):
        Ab, Pb = sh.block_rows(A, int(fb[r]), int(fb[r + 1])), sh.block_rows(P, int(fb[r]), int(fb[r + 1]))
        gens.append(sh.setup(OracleOps(), Ab, Pb, A.nrows, P.ncols, r, world, merged))
        vals.append((torch.as_tensor(Ab.val * (scale[r] if scale else 1.0)), torch.as_tensor(Pb.val)))
    return gens, vals


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


@pytest.mark.parametrize("kind", ["algebraic", "model"])
@pytest.mark.parametrize("merged", [True, False])
def test_lockstep_four_ranks(kind, merged):
    A, P = _problem(kind)
    world = 4
    gens, vals = _rank_gens(A, P, world, merged)
    plans = sh.run_lockstep(gens)
    assert all(p.remote_rows > 0 for p in plans)            # every block needs rows of P from others
    if not merged:
        assert all(len(p.parts) == 2 for p in plans)
    ops = OracleOps()
    outs = sh.run_lockstep([sh.numeric(ops, p, a, q) for p, (a, q) in zip(plans, vals)])
    for p, c in zip(plans, outs):
        _check_rows(A, P, p.c0, p.c1, p.own_rp, p.own_ci, c.numpy())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q, merged):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, P = _problem("algebraic")
        fb = pt.block_bounds(A.nrows, world)
        r0, r1 = int(fb[rank]), int(fb[rank + 1])
        Ab, Pb = sh.block_rows(A, r0, r1), sh.block_rows(P, r0, r1)   # all this rank holds
        del A, P
        comm = sh.TorchComm()
        ops = OracleOps()
        plan = sh.run(sh.setup(ops, Ab, Pb, fb[-1], Pb.ncols, rank, world, merged), comm)
        out = []
        for scale in (1.0, 0.5):     # a re-product with new values of A (same patterns)
            c = sh.run(sh.numeric(ops, plan, torch.as_tensor(Ab.val * scale), torch.as_tensor(Pb.val)), comm)
            out.append(c.numpy().copy())
        q.put((rank, plan.c0, plan.c1, plan.own_rp, plan.own_ci, out, plan.remote_rows))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,merged", [(2, True), (2, False), (3, False)])
def test_gloo_ranks(world, merged):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, merged)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert sorted(r[0] for r in res) == list(range(world))
    A, P = _problem("algebraic")
    for rank, c0, c1, own_rp, own_ci, outs, remote in res:
        assert remote > 0
        _check_rows(A, P, c0, c1, own_rp, own_ci, outs[0])
        _check_rows(A.with_values(A.val * 0.5), P, c0, c1, own_rp, own_ci, outs[1])
