"""Host logic of the multi-process row partition (Section 2, Eq. 1-3; Alg. 7-8).

Each process owns a contiguous block of fine rows of A and P (Eq. 1: n_l =
n / np rows, the remainder spread over the first processes) and the block of
coarse rows of C with the same rule over m.  Before its loop a process needs
the rows of P for the columns of its A block that other processes own (the
remote rows P~_r, gathered once per phase); after its loop it holds outer-
product contributions to coarse rows that other processes own (C_s), which it
sends to their owners, who add them (Alg. 7-8).

These functions are pure numpy on CSR arrays; one GPU per box here means the
exchange is exercised by CPU ranks (torch.distributed, gloo) in the tests.
"""
from __future__ import annotations

import numpy as np


def block_bounds(n: int, nranks: int) -> np.ndarray:
    """Row boundaries [b_0 = 0, ..., b_np = n] of the 1D block partition (Eq. 1)."""
    base, extra = divmod(n, nranks)
    sizes = np.full(nranks, base, dtype=np.int64)
    sizes[:extra] += 1
    return np.concatenate([[0], np.cumsum(sizes)])


def owner_of(idx: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Owning rank of each index under the block partition `bounds`."""
    return np.searchsorted(bounds, np.asarray(idx), side="right") - 1


def remote_rows(A, r0: int, r1: int) -> np.ndarray:
    """Sorted distinct columns of A(r0:r1, :) outside [r0, r1): the rows of P to fetch (P~_r)."""
    rp = np.asarray(A.row_ptr, dtype=np.int64)
    cols = np.asarray(A.col_idx[rp[r0]:rp[r1]])
    return np.unique(cols[(cols < r0) | (cols >= r1)])


def split_by_owner(rows: np.ndarray, row_ptr: np.ndarray, col_idx: np.ndarray, val: np.ndarray,
                   bounds: np.ndarray) -> dict:
    """Split partial coarse rows (CSR over `rows`) into per-owner messages.

    Returns {rank: (rows, row_ptr, col_idx, val)} for every rank that owns at
    least one of the rows.
    """
    rows = np.asarray(rows)
    rp = np.asarray(row_ptr, dtype=np.int64)
    own = owner_of(rows, bounds)
    out = {}
    for r in np.unique(own):
        sel = np.nonzero(own == r)[0]
        lens = rp[sel + 1] - rp[sel]
        idx = np.concatenate([np.arange(rp[s], rp[s + 1]) for s in sel]) if len(sel) else np.zeros(0, np.int64)
        out[int(r)] = (rows[sel], np.concatenate([[0], np.cumsum(lens)]), np.asarray(col_idx)[idx],
                       np.asarray(val)[idx])
    return out


def assemble(pieces, c0: int, c1: int):
    """Sum per-owner messages for the coarse rows [c0, c1) into CSR (columns sorted).

    The pattern is the union of the received patterns (structural: entries are
    kept even when their sum is zero).
    """
    acc: dict = {}
    for rows, rp, ci, v in pieces:
        for k, i in enumerate(rows):
            d = acc.setdefault(int(i) - c0, {})
            for e in range(int(rp[k]), int(rp[k + 1])):
                d[int(ci[e])] = d.get(int(ci[e]), 0.0) + float(v[e])
    n = c1 - c0
    lens = [len(acc.get(i, {})) for i in range(n)]
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cols, vals = [], []
    for i in range(n):
        d = acc.get(i, {})
        for j in sorted(d):
            cols.append(j)
            vals.append(d[j])
    return row_ptr, np.asarray(cols, dtype=np.int64), np.asarray(vals, dtype=np.float64)
