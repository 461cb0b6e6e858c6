"""The row-partitioned all-at-once product over processes (Section 2, Eq. 1-3;
Section 3, Alg. 7-10), one process per GPU.

Process r owns the fine rows [r0, r1) of A and P (Eq. 1) and the coarse rows
[c0, c1) of C (the same rule over m).  Its block of the product is

    C_r = sum over I in [r0, r1) of P(I,:)^T (x) (A(I,:) P)            (Eq. 9)

which needs the rows of P that A(r0:r1, :) references outside [r0, r1) --
the remote rows P~_r, gathered from their owners once per phase -- and which
touches coarse rows other processes own (C_s), sent to those owners and added
there.  Locally the block is an ordinary square triple product: with the
fine rows renumbered [own rows | remote rows], A_sq holds A's block in its
first n_l rows (empty rows after), P_ext holds [P(r0:r1, :); P~_r], and
P_ext^T A_sq P_ext is exactly C_r, so the library's symbolic and numeric
phases run unchanged on it.

Setup (the symbolic phase, Alg. 7) exchanges patterns once: the remote row
requests, the pattern of those P rows, and the pattern of the C_s rows; it
fixes every index list of the numeric phase.  A numeric phase (Alg. 8)
moves values only:

  1. pack the P values other processes requested, exchange, place them
     after the own rows of P_ext (the sparse update of P~_r);
  2. permute A's block values into A_sq's column order;
  3. run the local product(s);
  4. pack the C_s values, exchange, and add own and received values into the
     owned rows of C (zeroed first).

``merged=True`` runs one local product over all own fine rows, then sends
C_s (the merged loop of Alg. 9-10).  ``merged=False`` is the remote-first
loop of Alg. 7-8: the fine rows whose P(I,:) reaches a coarse row owned
elsewhere go first, their C_s is sent while the remaining (purely local)
rows run.  Both give the same C.

The value movement and the local products are delegated to a backend
(``LibraryOps``: the CUDA library, one GPU per process; tests also supply an
oracle-backed one for CPU ranks) and the exchanges to a communicator
(``TorchComm``: torch.distributed point-to-point, NCCL on GPUs or gloo on
CPUs).  Everything here runs once per setup or marshals a few index lists.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import partition as pt


# ---------------------------------------------------------------------------
# communicator
# ---------------------------------------------------------------------------
class TorchComm:
    """Personalised exchange over torch.distributed point-to-point calls.

    ``exchange(send)`` sends send[d] to rank d and returns recv[s] from every
    rank s (recv[rank] = send[rank]).  Sizes are exchanged first unless the
    caller passes the receive sizes (fixed after setup).
    """

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _sizes(self, send):
        dist = self.dist
        mine = torch.tensor([int(t.numel()) for t in send], dtype=torch.int64)
        if send and send[0].is_cuda:
            mine = mine.to(send[0].device)
        allsz = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(allsz, mine, group=self.group)
        return [int(a[self.rank]) for a in allsz]

    def start(self, send, recv_sizes=None, dtype=None):
        """Posts the exchange; returns (recv buffers, handles) -- wait() on the handles."""
        dist = self.dist
        if recv_sizes is None:
            recv_sizes = self._sizes(send)
        ref = send[self.rank]
        recv = [torch.empty(n, dtype=dtype or ref.dtype, device=ref.device) for n in recv_sizes]
        recv[self.rank] = send[self.rank]
        ops = []
        for k in range(1, self.world):
            d = (self.rank + k) % self.world       # send to d while receiving from s
            s = (self.rank - k) % self.world
            if send[d].numel():
                ops.append(dist.isend(send[d].contiguous(), d, group=self.group))
            if recv[s].numel():
                ops.append(dist.irecv(recv[s], s, group=self.group))
        return recv, ops

    def exchange(self, send, recv_sizes=None):
        recv, ops = self.start(send, recv_sizes)
        for op in ops:
            op.wait()
        return recv


# ---------------------------------------------------------------------------
# exchange protocol: setup and numeric are generators that yield their
# exchanges, so that one rank per process (``run``) and all ranks stepped in
# lockstep in one process (``run_lockstep``) drive the same code
# ---------------------------------------------------------------------------
@dataclass
class Exchange:
    send: list                      # send[d]: tensor for rank d
    recv_sizes: list | None = None  # known receive sizes (fixed after setup)
    recv_into: list | None = None   # receive buffers to fill (views allowed), else allocated
    wait: bool = True               # False: returns a handle that a later Wait completes


@dataclass
class Wait:
    handle: object


def run(gen, comm: TorchComm):
    """Drives one rank's setup or numeric generator with a real communicator."""
    try:
        msg = next(gen)
        while True:
            if isinstance(msg, Exchange):
                recv, ops = comm.start(msg.send, msg.recv_sizes)
                if msg.wait:
                    for op in ops:
                        op.wait()
                    res = _fill(recv, msg.recv_into, comm.rank)
                else:
                    res = (recv, ops, msg.recv_into)
            else:
                recv, ops, into = msg.handle
                for op in ops:
                    op.wait()
                res = _fill(recv, into, comm.rank)
            msg = gen.send(res)
    except StopIteration as stop:
        return stop.value


def _fill(recv, into, rank):
    if into is None:
        return recv
    for s, (r, b) in enumerate(zip(recv, into)):
        if b is not None and s != rank and r.numel():
            b.copy_(r)
    return into


def run_lockstep(gens):
    """Drives the generators of all ranks in one process, phase by phase; exchanges
    are list transpositions.  For tests on CPU and for ranks emulated one after the
    other on one GPU (no kernel of one rank ever waits for another's)."""
    world = len(gens)
    msgs = [next(g) for g in gens]
    results = [None] * world
    while True:
        kinds = {type(m) for m in msgs}
        assert len(kinds) == 1, "ranks diverged"
        if isinstance(msgs[0], Exchange):
            res = []
            for r in range(world):
                recv = [msgs[s].send[r].clone() if s != r else msgs[r].send[r] for s in range(world)]
                res.append(_fill(recv, msgs[r].recv_into, r))
        else:
            res = [m.handle for m in msgs]
        nxt = []
        done = 0
        for r, g in enumerate(gens):
            try:
                if isinstance(msgs[r], Exchange) and not msgs[r].wait:
                    nxt.append(g.send(res[r]))       # the handle is the completed exchange
                else:
                    nxt.append(g.send(res[r]))
            except StopIteration as stop:
                results[r] = stop.value
                nxt.append(None)
                done += 1
        if done == world:
            return results
        assert done == 0, "ranks diverged"
        msgs = nxt


# ---------------------------------------------------------------------------
# the rank's plan
# ---------------------------------------------------------------------------
@dataclass
class Part:
    """One local product: the own fine rows `rows` of the block in A_sq."""
    plan: object
    a_perm: object        # positions in the block's A values, in A_sq's entry order
    c_rp: np.ndarray      # pattern of this part's C_r (m rows)
    c_ci: np.ndarray
    c_vals: object = None
    own_src: object = None   # positions in c_vals of entries in owned coarse rows
    own_dst: object = None   # their positions in the owned rows of C


@dataclass
class RankPlan:
    rank: int
    world: int
    r0: int
    r1: int
    c0: int
    c1: int
    merged: bool
    n_ext: int
    p_send_idx: list = field(default_factory=list)   # per rank: positions in the block's P values
    p_recv_sizes: list = field(default_factory=list)
    p_recv_off: list = field(default_factory=list)   # per rank: offset of its rows' values in P_ext
    p_nnz_local: int = 0
    p_ext_nnz: int = 0
    parts: list = field(default_factory=list)
    c_send_idx: list = field(default_factory=list)   # per rank: positions in parts[0].c_vals
    c_recv_sizes: list = field(default_factory=list)
    recv_dst: list = field(default_factory=list)     # per rank: positions in the owned rows of C
    own_rp: np.ndarray = None                        # pattern of the owned rows [c0, c1) of C
    own_ci: np.ndarray = None
    remote_rows: int = 0
    p_ext_vals: object = None
    c_own: object = None


def _ranges(rp, rows):
    """Concatenated index ranges [rp[i], rp[i+1]) for i in rows."""
    rp = np.asarray(rp, dtype=np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    lens = rp[rows + 1] - rp[rows]
    if lens.sum() == 0:
        return np.zeros(0, dtype=np.int64)
    starts = np.repeat(rp[rows] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return starts + np.arange(int(lens.sum()), dtype=np.int64)


def _csr(nrows, ncols, rp, ci):
    from .problems import CSR
    rp = np.asarray(rp, dtype=np.int64)
    return CSR(int(nrows), int(ncols), rp.astype(np.int32), np.asarray(ci, dtype=np.int32),
               np.zeros(len(ci)))


def setup(ops, A_blk, P_blk, n: int, m: int, rank: int, world: int, merged: bool = True):
    """Symbolic phase of the rank's block (Alg. 7), as a generator of exchanges.

    A_blk / P_blk: host CSR of the rank's fine rows [r0, r1) of A (global
    columns) and P.  Returns the RankPlan.
    """
    fb, cb = pt.block_bounds(n, world), pt.block_bounds(m, world)
    r0, r1, c0, c1 = int(fb[rank]), int(fb[rank + 1]), int(cb[rank]), int(cb[rank + 1])
    n_l = r1 - r0
    assert A_blk.nrows == n_l and P_blk.nrows == n_l
    a_rp = np.asarray(A_blk.row_ptr, dtype=np.int64)
    a_ci = np.asarray(A_blk.col_idx, dtype=np.int64)
    p_rp = np.asarray(P_blk.row_ptr, dtype=np.int64)
    p_ci = np.asarray(P_blk.col_idx, dtype=np.int64)
    # remote rows of P this block references, grouped by owner (ascending ids)
    remote = np.unique(a_ci[(a_ci < r0) | (a_ci >= r1)])
    owner = pt.owner_of(remote, fb)
    req = [remote[owner == d] for d in range(world)]
    want = yield Exchange([ops.comm_i64(x) for x in req])
    want = [ops.np(w) for w in want]
    want[rank] = np.zeros(0, dtype=np.int64)
    # the pattern of the requested rows: lengths, then columns
    lens_out = [p_rp[w - r0 + 1] - p_rp[w - r0] if len(w) else np.zeros(0, np.int64) for w in want]
    idx_out = [_ranges(p_rp, w - r0) for w in want]
    lens_in = yield Exchange([ops.comm_i64(x) for x in lens_out])
    cols_in = yield Exchange([ops.comm_i64(p_ci[x]) for x in idx_out])
    lens_in = [ops.np(x) for x in lens_in]
    cols_in = [ops.np(x) for x in cols_in]
    lens_in[rank] = np.zeros(0, np.int64)
    cols_in[rank] = np.zeros(0, np.int64)
    rp_plan = RankPlan(rank, world, r0, r1, c0, c1, merged, n_l + len(remote))
    rp_plan.remote_rows = int(len(remote))
    rp_plan.p_send_idx = [ops.index(x) for x in idx_out]
    rp_plan.p_recv_sizes = [int(len(x)) for x in cols_in]
    rp_plan.p_nnz_local = int(p_rp[-1])
    off = rp_plan.p_nnz_local
    for d in range(world):
        rp_plan.p_recv_off.append(off)
        off += len(cols_in[d])
    rp_plan.p_ext_nnz = off
    # P_ext = [P(r0:r1, :); P~_r]
    ext_lens = np.concatenate([np.diff(p_rp)] + [lens_in[d] for d in range(world)])
    P_ext = _csr(rp_plan.n_ext, m, np.concatenate([[0], np.cumsum(ext_lens)]),
                 np.concatenate([p_ci] + [cols_in[d] for d in range(world)]))
    # A_sq: own rows renumbered 0..n_l-1, remote rows n_l..; each row's entries sorted
    newc = np.where((a_ci >= r0) & (a_ci < r1), a_ci - r0, n_l + np.searchsorted(remote, a_ci))
    row_of = np.repeat(np.arange(n_l, dtype=np.int64), np.diff(a_rp))
    perm = np.lexsort((newc, row_of))
    newc, row_of = newc[perm], row_of[perm]
    # fine rows whose P(I,:) reaches a coarse row owned elsewhere (the remote part of Alg. 7-8)
    p_row_of = np.repeat(np.arange(n_l, dtype=np.int64), np.diff(p_rp))
    far = np.zeros(n_l, dtype=bool)
    far[p_row_of[(p_ci < c0) | (p_ci >= c1)]] = True
    selections = [np.ones(n_l, dtype=bool)] if merged else [far, ~far]
    for sel in selections:
        keep = sel[row_of]
        lens = np.bincount(row_of[keep], minlength=rp_plan.n_ext)
        A_part = _csr(rp_plan.n_ext, rp_plan.n_ext, np.concatenate([[0], np.cumsum(lens)]), newc[keep])
        plan, c_rp, c_ci = ops.plan(A_part, P_ext)
        rp_plan.parts.append(Part(plan, ops.index(perm[keep]), np.asarray(c_rp, np.int64),
                                  np.asarray(c_ci, np.int64)))
    # C_s: rows of the first part (merged: all; remote-first: the far rows) owned elsewhere
    first = rp_plan.parts[0]
    nz_rows = np.nonzero(np.diff(first.c_rp))[0]
    s_rows = nz_rows[(nz_rows < c0) | (nz_rows >= c1)]
    s_owner = pt.owner_of(s_rows, cb)
    c_rows_out = [s_rows[s_owner == d] for d in range(world)]
    c_idx_out = [_ranges(first.c_rp, x) for x in c_rows_out]
    for part in rp_plan.parts[1:]:
        rows = np.nonzero(np.diff(part.c_rp))[0]
        assert np.all((rows >= c0) & (rows < c1)), "purely local rows reached a remote coarse row"
    rows_in = yield Exchange([ops.comm_i64(x) for x in c_rows_out])
    lens_in = yield Exchange([ops.comm_i64(np.diff(first.c_rp)[x]) for x in c_rows_out])
    cols_in = yield Exchange([ops.comm_i64(first.c_ci[x]) for x in c_idx_out])
    rows_in = [ops.np(x) for x in rows_in]
    lens_in = [ops.np(x) for x in lens_in]
    cols_in = [ops.np(x) for x in cols_in]
    for x in (rows_in, lens_in, cols_in):
        x[rank] = np.zeros(0, np.int64)
    rp_plan.c_send_idx = [ops.index(x) for x in c_idx_out]
    rp_plan.c_recv_sizes = [int(len(x)) for x in cols_in]
    # owned rows of C: the union of every contribution's pattern (structural)
    keys_src = []
    for part in rp_plan.parts:
        rows = np.arange(c0, c1, dtype=np.int64)
        idx = _ranges(part.c_rp, rows)
        r_of = np.repeat(rows, part.c_rp[rows + 1] - part.c_rp[rows])
        keys_src.append(("own", part, idx, (r_of - c0) * m + part.c_ci[idx]))
    for s in range(world):
        r_of = np.repeat(rows_in[s], lens_in[s])
        keys_src.append(("recv", s, None, (r_of - c0) * m + cols_in[s]))
    keys = np.unique(np.concatenate([k[3] for k in keys_src])) if keys_src else np.zeros(0, np.int64)
    rows_own = keys // m
    rp_plan.own_rp = np.concatenate([[0], np.cumsum(np.bincount(rows_own, minlength=c1 - c0))]).astype(np.int64)
    rp_plan.own_ci = (keys % m).astype(np.int64)
    rp_plan.recv_dst = [None] * world
    for kind, who, idx, k in keys_src:
        dst = ops.index(np.searchsorted(keys, k))
        if kind == "own":
            who.own_src, who.own_dst = ops.index(idx), dst
        else:
            rp_plan.recv_dst[who] = dst
    ops.allocate(rp_plan)
    return rp_plan


def numeric(ops, plan: RankPlan, A_vals, P_vals):
    """Numeric phase of the rank's block (Alg. 8; merged loop of Alg. 9-10 when
    plan.merged), as a generator of exchanges.  A_vals / P_vals: the values of the
    rank's blocks of A and P (backend tensors, block CSR order).  Returns the
    values of the owned rows of C (pattern plan.own_rp / plan.own_ci)."""
    world, rank = plan.world, plan.rank
    # 1. the sparse update of P~_r: pack what others requested, receive into P_ext
    send = [ops.gather(P_vals, plan.p_send_idx[d]) if d != rank else ops.empty(0) for d in range(world)]
    into = [plan.p_ext_vals[plan.p_recv_off[s]:plan.p_recv_off[s] + plan.p_recv_sizes[s]]
            if s != rank else None for s in range(world)]
    pending = yield Exchange(send, plan.p_recv_sizes, into, wait=False)
    ops.copy(plan.p_ext_vals[:plan.p_nnz_local], P_vals)   # own rows while the halo is in flight
    yield Wait(pending)
    # 2-3. local products; C_s is packed after the first part and exchanged while the
    # second (purely local) part runs in the remote-first loop
    first = plan.parts[0]
    ops.numeric(first.plan, ops.gather(A_vals, first.a_perm), plan.p_ext_vals, first.c_vals)
    send = [ops.gather(first.c_vals, plan.c_send_idx[d]) if d != rank else ops.empty(0) for d in range(world)]
    pending = yield Exchange(send, plan.c_recv_sizes, wait=False)
    for part in plan.parts[1:]:
        ops.numeric(part.plan, ops.gather(A_vals, part.a_perm), plan.p_ext_vals, part.c_vals)
    recv = yield Wait(pending)
    # 4. owned rows of C: own contributions and the received C_s, added at fixed positions
    ops.zero(plan.c_own)
    for part in plan.parts:
        ops.scatter_add(plan.c_own, part.own_dst, part.c_vals, part.own_src)
    for s in range(world):
        if s != rank and plan.c_recv_sizes[s]:
            ops.scatter_add(plan.c_own, plan.recv_dst[s], recv[s])
    return plan.c_own


# ---------------------------------------------------------------------------
# backend: the CUDA library, one GPU per process
# ---------------------------------------------------------------------------
class LibraryOps:
    """Local products (ptap_symbolic / ptap_numeric on A_sq and P_ext) and value
    movement (ptap_gather / ptap_scatter_add) on one GPU."""

    def __init__(self, device, dtype=torch.float64, config=None):
        from . import ptap
        self.ptap = ptap
        self.device = torch.device(device)
        self.dtype = dtype
        self.config = config
        self._pat = {}

    # setup-time conversions (patterns travel as int64 tensors on the device)
    def comm_i64(self, x):
        return torch.as_tensor(np.asarray(x, dtype=np.int64)).to(self.device)

    def np(self, t):
        return t.cpu().numpy().astype(np.int64)

    def index(self, x):
        return torch.as_tensor(np.asarray(x, dtype=np.int64).astype(np.int32)).to(self.device)

    def plan(self, A_part, P_ext):
        ptap = self.ptap
        dA = ptap.Csr.from_host(A_part, self.device, self.dtype)
        dP = ptap.Csr.from_host(P_ext, self.device, self.dtype)
        plan = ptap.symbolic(dA, dP, self.config)
        rp, ci = plan.pattern()
        self._pat[id(plan)] = (dA, dP)
        return plan, rp.cpu().numpy(), ci.cpu().numpy()

    def allocate(self, rp_plan):
        rp_plan.p_ext_vals = torch.empty(rp_plan.p_ext_nnz, dtype=self.dtype, device=self.device)
        for part in rp_plan.parts:
            part.c_vals = torch.empty(part.plan.nnz, dtype=self.dtype, device=self.device)
        rp_plan.c_own = torch.empty(int(rp_plan.own_rp[-1]), dtype=self.dtype, device=self.device)

    # numeric-time value movement and products
    def empty(self, n):
        return torch.empty(n, dtype=self.dtype, device=self.device)

    def gather(self, src, idx):
        return self.ptap.gather(src, idx) if idx.numel() else self.empty(0)

    def scatter_add(self, dst, dst_idx, src, src_idx=None):
        if dst_idx.numel():
            self.ptap.scatter_add(dst, dst_idx, src, src_idx)

    def copy(self, dst, src):
        dst.copy_(src)

    def zero(self, t):
        t.zero_()

    def numeric(self, plan, A_vals, P_vals, out):
        dA, dP = self._pat[id(plan)]
        self.ptap.numeric(plan, dA.with_values(A_vals), dP.with_values(P_vals), out)


def block_rows(M, r0: int, r1: int):
    """Host CSR of rows [r0, r1) of M (global column indices kept)."""
    from .problems import CSR
    rp = np.asarray(M.row_ptr, dtype=np.int64)
    a, b = int(rp[r0]), int(rp[r1])
    return CSR(r1 - r0, M.ncols, (rp[r0:r1 + 1] - a).astype(np.int32), np.asarray(M.col_idx[a:b]),
               np.asarray(M.val[a:b]))
