"""Seeded synthetic inputs for the sparse triple product C = P^T A P.

This module builds fine-level operators A and interpolation operators P in CSR
form (int32 indices, float64 values).  It holds none of the triple product's
arithmetic: the oracle and the CUDA path both take their inputs from here and
from nowhere else.

Workloads (the paper's own matrices are not public; these stand in for them):

* Model problem (Section 4.1): a 3D Laplacian on a structured grid with linear
  (trilinear) interpolation from a coarse grid of half the resolution.  The
  paper's grids include boundary vertices (fine 1999 / coarse 1000); here the
  boundary is Dirichlet and eliminated, so a fine interior side n maps to a
  coarse interior side n // 2 (fine point 2j sits on coarse point j).
* Algebraic case (Section 4.2, Tables 5-6 row statistics): a 27-point operator
  with lognormal edge weights and a smoothed-aggregation P.
* A 2D 5-point Poisson operator with a smoothed-aggregation P.
* Tiny random matrices with explicit zeros and empty rows/columns.

Grid points are ordered lexicographically with x fastest:
``index = x + nx * (y + ny * z)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Compressed sparse row matrix with sorted, unique column indices per row."""

    nrows: int
    ncols: int
    row_ptr: np.ndarray  # int32 [nrows + 1]
    col_idx: np.ndarray  # int32 [nnz]
    val: np.ndarray      # float64 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astype(self, dtype) -> "CSR":
        return CSR(self.nrows, self.ncols, self.row_ptr, self.col_idx,
                   np.ascontiguousarray(self.val.astype(dtype)))

    def with_values(self, val: np.ndarray) -> "CSR":
        assert val.shape == self.col_idx.shape
        return CSR(self.nrows, self.ncols, self.row_ptr, self.col_idx,
                   np.ascontiguousarray(val))

    def abs(self) -> "CSR":
        return self.with_values(np.abs(self.val))

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=np.float64)
        rows = np.repeat(np.arange(self.nrows), self.row_lengths())
        np.add.at(d, (rows, self.col_idx), self.val.astype(np.float64))
        return d

    def pattern_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=bool)
        rows = np.repeat(np.arange(self.nrows), self.row_lengths())
        d[rows, self.col_idx] = True
        return d

    def check(self) -> None:
        """Raise if the CSR invariants (int32, monotone, sorted unique cols) fail."""
        assert self.row_ptr.dtype == np.int32 and self.col_idx.dtype == np.int32
        assert self.row_ptr.shape == (self.nrows + 1,) and self.row_ptr[0] == 0
        lens = self.row_lengths()
        assert (lens >= 0).all()
        assert self.col_idx.shape == (self.nnz,) and self.val.shape == (self.nnz,)
        if self.nnz:
            assert self.col_idx.min() >= 0 and self.col_idx.max() < self.ncols
            d = np.diff(self.col_idx.astype(np.int64))
            starts = np.zeros(self.nnz, dtype=bool)
            starts[self.row_ptr[:-1][lens > 0]] = True
            assert (d[~starts[1:]] > 0).all(), "columns must be sorted and unique"


def csr_from_slots(cols: np.ndarray, vals: np.ndarray, valid: np.ndarray,
                   ncols: int) -> CSR:
    """Build CSR from per-row slot arrays of shape [nslots, nrows].

    Slots must already be in ascending column order within each row.
    """
    nslots, nrows = valid.shape
    lens = valid.sum(axis=0, dtype=np.int64)
    row_ptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    assert row_ptr[-1] < 2**31, "nnz must fit int32 indexing"
    vt = np.ascontiguousarray(valid.T)
    col_idx = np.ascontiguousarray(cols.T)[vt].astype(np.int32)
    val = np.ascontiguousarray(vals.T)[vt].astype(np.float64)
    return CSR(nrows, ncols, row_ptr.astype(np.int32), col_idx, val)


# --------------------------------------------------------------------------
# structured-grid operators in stencil form
# --------------------------------------------------------------------------

def _axis_valid(n: int, d: int) -> np.ndarray:
    x = np.arange(n)
    return (x + d >= 0) & (x + d < n)


def _grid_valid(shape, off) -> np.ndarray:
    nz, ny, nx = shape
    dz, dy, dx = off
    v = (_axis_valid(nz, dz)[:, None, None] & _axis_valid(ny, dy)[None, :, None]
         & _axis_valid(nx, dx)[None, None, :])
    return v.reshape(-1)


@dataclass
class Stencil:
    """Grid operator: for each offset o and point p, value vals[o, p] if valid[o, p]."""

    shape: tuple          # (nz, ny, nx)
    offsets: list         # [(dz, dy, dx)] in ascending linear-offset order
    vals: np.ndarray      # float64 [noff, npts]
    valid: np.ndarray     # bool    [noff, npts]

    @property
    def npts(self) -> int:
        nz, ny, nx = self.shape
        return nz * ny * nx

    def lin(self, off) -> int:
        nz, ny, nx = self.shape
        dz, dy, dx = off
        return dx + nx * (dy + ny * dz)

    def to_csr(self) -> CSR:
        n = self.npts
        idx = np.arange(n, dtype=np.int64)
        cols = np.empty((len(self.offsets), n), dtype=np.int64)
        for o, off in enumerate(self.offsets):
            cols[o] = idx + self.lin(off)
        cols[~self.valid] = 0
        return csr_from_slots(cols, self.vals, self.valid, n)

    def diagonal(self) -> np.ndarray:
        return self.vals[self.offsets.index((0, 0, 0))]


def _sorted_offsets(offs, shape):
    nz, ny, nx = shape
    return sorted(offs, key=lambda o: o[2] + nx * (o[1] + ny * o[0]))


def laplacian_7pt(n: int | tuple) -> Stencil:
    """3D 7-point Laplacian: 6 on the diagonal, -1 off it, Dirichlet neighbours dropped."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    offs = _sorted_offsets([(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                            (0, 0, -1), (0, 0, 1)], shape)
    npts = shape[0] * shape[1] * shape[2]
    vals = np.empty((len(offs), npts))
    valid = np.empty((len(offs), npts), dtype=bool)
    for o, off in enumerate(offs):
        valid[o] = _grid_valid(shape, off)
        vals[o] = 6.0 if off == (0, 0, 0) else -1.0
    return Stencil(shape, offs, vals, valid)


def laplacian_5pt_2d(n: int) -> Stencil:
    """2D 5-point Poisson operator (4 on the diagonal, -1 off it), Dirichlet."""
    shape = (1, n, n)
    offs = _sorted_offsets([(0, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)], shape)
    npts = n * n
    vals = np.empty((len(offs), npts))
    valid = np.empty((len(offs), npts), dtype=bool)
    for o, off in enumerate(offs):
        valid[o] = _grid_valid(shape, off)
        vals[o] = 4.0 if off == (0, 0, 0) else -1.0
    return Stencil(shape, offs, vals, valid)


def laplacian_27pt_lognormal(n: int | tuple, seed: int, neumann: bool = False) -> Stencil:
    """27-point graph Laplacian with one lognormal(0,1) weight per undirected edge.

    A(p, q) = -w_pq for the 26 neighbours q inside the grid and
    A(p, p) = sum of w over all 26 edges of p.  With ``neumann=False`` the edges
    to eliminated points outside the grid still count on the diagonal (rows on
    the boundary are strictly diagonally dominant, interior rows sum to zero).
    With ``neumann=True`` only edges inside the grid count, so every row sums
    to zero.  Weights are drawn on the grid extended by one layer, indexed by
    the edge's lexicographically lower endpoint, so each edge has exactly one
    weight and A is symmetric.
    """
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    pos_dirs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dz, dy, dx) > (0, 0, 0)]
    assert len(pos_dirs) == 13
    W = rng.lognormal(0.0, 1.0, size=(13, nz + 2, ny + 2, nx + 2))
    offs = _sorted_offsets([(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
                            for dx in (-1, 0, 1)], shape)
    npts = nz * ny * nx
    vals = np.zeros((27, npts))
    valid = np.empty((27, npts), dtype=bool)
    diag = np.zeros(npts)
    for o, off in enumerate(offs):
        valid[o] = _grid_valid(shape, off)
        if off == (0, 0, 0):
            continue
        if off > (0, 0, 0):
            d = pos_dirs.index(off)
            s = (1, 1, 1)
        else:
            d = pos_dirs.index((-off[0], -off[1], -off[2]))
            s = (1 + off[0], 1 + off[1], 1 + off[2])
        w = W[d, s[0]:s[0] + nz, s[1]:s[1] + ny, s[2]:s[2] + nx].reshape(-1)
        vals[o] = -w
        if neumann:
            diag += np.where(valid[o], w, 0.0)
        else:
            diag += w
    vals[offs.index((0, 0, 0))] = diag
    vals[~valid] = 0.0
    return Stencil(shape, offs, vals, valid)


# --------------------------------------------------------------------------
# interpolation operators
# --------------------------------------------------------------------------

def _linear_1d(n: int):
    """1D linear interpolation from coarse interior side n // 2 to fine side n.

    Fine point X (1-based, 1..n): X = 2j takes weight 1 from coarse j;
    X = 2j+1 takes 1/2 from coarse j and j+1 where those lie in 1..n//2.
    Returns (cand[2, n], wgt[2, n], present[2, n]) with 0-based coarse indices,
    slot 0 holding the lower index.
    """
    if n == 1:   # a one-point axis is not coarsened
        return (np.zeros((2, 1), np.int64), np.array([[1.0], [0.0]]),
                np.array([[True], [False]]), 1)
    md = n // 2
    X = np.arange(1, n + 1)
    cand = np.zeros((2, n), dtype=np.int64)
    wgt = np.zeros((2, n))
    pres = np.zeros((2, n), dtype=bool)
    even = X % 2 == 0
    cand[0, even] = X[even] // 2 - 1
    wgt[0, even] = 1.0
    pres[0, even] = True
    odd = ~even
    lo = (X[odd] - 1) // 2 - 1
    hi = lo + 1
    lo_ok = lo >= 0
    hi_ok = hi < md
    # lower slot: lo if present, else hi
    c0 = np.where(lo_ok, lo, hi)
    p0 = lo_ok | hi_ok
    c1 = hi
    p1 = lo_ok & hi_ok
    cand[0, odd] = c0
    wgt[0, odd] = 0.5
    pres[0, odd] = p0
    cand[1, odd] = c1
    wgt[1, odd] = 0.5
    pres[1, odd] = p1
    return cand, wgt, pres, md


def trilinear_P(n: int | tuple) -> CSR:
    """Tensor-product linear interpolation (weights 1, 1/2, 1/4, 1/8) on an n^3 grid."""
    shape = (n, n, n) if isinstance(n, int) else tuple(n)
    nz, ny, nx = shape
    cz, wz, pz, mz = _linear_1d(nz)
    cy, wy, py, my = _linear_1d(ny)
    cx, wx, px, mx = _linear_1d(nx)
    npts = nz * ny * nx
    cols = np.empty((8, npts), dtype=np.int64)
    vals = np.empty((8, npts))
    valid = np.empty((8, npts), dtype=bool)
    s = 0
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                c = (cx[bx][None, None, :] + mx * (cy[by][None, :, None] + my * cz[bz][:, None, None]))
                w = wx[bx][None, None, :] * wy[by][None, :, None] * wz[bz][:, None, None]
                v = px[bx][None, None, :] & py[by][None, :, None] & pz[bz][:, None, None]
                cols[s] = c.reshape(-1)
                vals[s] = w.reshape(-1)
                valid[s] = v.reshape(-1)
                s += 1
    cols[~valid] = 0
    P = csr_from_slots(cols, vals, valid, mx * my * mz)
    return P


def _aggregates_1d(n: int, w: int):
    """Aggregate id per fine point along one axis: boxes of width w.

    A trailing remainder of 1 point is merged into the previous box, so every
    box is at least 2 wide and a point's neighbours span at most 2 boxes.
    """
    if n <= w:
        na = 1
    else:
        na = n // w + (1 if n % w >= 2 else 0)
    agg = np.minimum(np.arange(n) // w, na - 1)
    return agg, na


def smoothed_aggregation_P(A: Stencil, widths: tuple, omega: float = 2.0 / 3.0) -> CSR:
    """P = (I - omega D^-1 A) T with T the unnormalised box-aggregation operator.

    T(p, agg(p)) = 1, so T maps constants to constants.  The pattern of P is
    structural: pat(A) pat(T) (which contains pat(T) since A has a full
    diagonal); entries that happen to evaluate to zero are kept.
    """
    nz, ny, nx = A.shape
    wz, wy, wx = widths
    az, naz = _aggregates_1d(nz, wz)
    ay, nay = _aggregates_1d(ny, wy)
    ax, nax = _aggregates_1d(nx, wx)

    def cand(agg, n):
        lo = agg[np.maximum(np.arange(n) - 1, 0)]
        hi = agg[np.minimum(np.arange(n) + 1, n - 1)]
        return lo, hi

    loz, hiz = cand(az, nz)
    loy, hiy = cand(ay, ny)
    lox, hix = cand(ax, nx)
    npts = nz * ny * nx
    acc = np.zeros((8, npts))
    pres = np.zeros((8, npts), dtype=bool)
    zz = np.arange(nz)
    yy = np.arange(ny)
    xx = np.arange(nx)
    for o, (dz, dy, dx) in enumerate(A.offsets):
        bz = (az[np.clip(zz + dz, 0, nz - 1)] != loz).astype(np.int64)
        by = (ay[np.clip(yy + dy, 0, ny - 1)] != loy).astype(np.int64)
        bx = (ax[np.clip(xx + dx, 0, nx - 1)] != lox).astype(np.int64)
        combo = (bz[:, None, None] * 4 + by[None, :, None] * 2 + bx[None, None, :]).reshape(-1)
        v = A.valid[o]
        a = np.where(v, A.vals[o], 0.0)
        for c in range(8):
            m = v & (combo == c)
            acc[c] += np.where(m, a, 0.0)
            pres[c] |= m
    # delta term: the point's own aggregate
    bz = (az != loz).astype(np.int64)
    by = (ay != loy).astype(np.int64)
    bx = (ax != lox).astype(np.int64)
    self_combo = (bz[:, None, None] * 4 + by[None, :, None] * 2 + bx[None, None, :]).reshape(-1)
    diag = A.diagonal()
    scale = omega / diag
    cols = np.empty((8, npts), dtype=np.int64)
    vals = np.empty((8, npts))
    for c in range(8):
        sz, sy, sx = (c >> 2) & 1, (c >> 1) & 1, c & 1
        gz = np.where(sz, hiz, loz)
        gy = np.where(sy, hiy, loy)
        gx = np.where(sx, hix, lox)
        cols[c] = (gx[None, None, :] + nax * (gy[None, :, None] + nay * gz[:, None, None])).reshape(-1)
        vals[c] = (self_combo == c).astype(np.float64) - scale * acc[c]
        pres[c] |= self_combo == c
    cols[~pres] = 0
    return csr_from_slots(cols, vals, pres, naz * nay * nax)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def model_problem(n: int):
    """7-point Laplacian on n^3 with trilinear P to (n//2)^3 (Section 4.1 model problem)."""
    A = laplacian_7pt(n).to_csr()
    P = trilinear_P(n)
    return A, P


def algebraic_problem(n: int, seed: int = 3, agg: int = 3, neumann: bool = False):
    """27-point lognormal operator on n^3 with smoothed-aggregation P (agg^3 boxes)."""
    S = laplacian_27pt_lognormal(n, seed, neumann=neumann)
    P = smoothed_aggregation_P(S, (agg, agg, agg))
    return S.to_csr(), P


def poisson2d_problem(n: int, agg: int = 2):
    """2D 5-point Poisson on n^2 with smoothed-aggregation P (agg x agg boxes)."""
    S = laplacian_5pt_2d(n)
    P = smoothed_aggregation_P(S, (1, agg, agg))
    return S.to_csr(), P


def batch_problems(seed: int = 4, count: int = 64, lo: int = 16, hi: int = 96):
    """Uneven batch: sides ~ U{lo..hi}; stencil and P type alternate.

    Problem k uses a 7-point operator if k is even, else a 27-point lognormal
    one (seed 1000 + k); P is trilinear if (k // 2) is even, else smoothed
    aggregation with 3^3 boxes.
    """
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=count)
    out = []
    for k, n in enumerate(sides):
        n = int(n)
        S = laplacian_7pt(n) if k % 2 == 0 else laplacian_27pt_lognormal(n, 1000 + k)
        if (k // 2) % 2 == 0:
            P = trilinear_P(n)
        else:
            P = smoothed_aggregation_P(S, (3, 3, 3))
        out.append((S.to_csr(), P))
    return out


def rescale_values(M: CSR, seed: int, lo: float = 0.5, hi: float = 2.0) -> CSR:
    """Per-entry i.i.d. uniform(lo, hi) rescale of the stored values (pattern fixed)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(lo, hi, size=M.nnz)
    return M.with_values(M.val * f)


def perturb_values(M: CSR, seed: int, sigma: float = 0.05) -> CSR:
    """Add N(0, sigma^2) noise to the stored values (pattern fixed)."""
    rng = np.random.default_rng(seed)
    return M.with_values(M.val + rng.normal(0.0, sigma, size=M.nnz))


def random_csr(nrows: int, ncols: int, density: float, rng: np.random.Generator,
               int_values: bool = True, zero_frac: float = 0.1,
               empty_row_frac: float = 0.1) -> CSR:
    """Random CSR with explicit stored zeros and some empty rows.

    Values are small integers (exact in float32 and float64 arithmetic) when
    ``int_values`` is set, else standard normal.
    """
    mask = rng.random((nrows, ncols)) < density
    empty = rng.random(nrows) < empty_row_frac
    mask[empty] = False
    rows, cols = np.nonzero(mask)
    if int_values:
        vals = rng.integers(-3, 4, size=rows.size).astype(np.float64)
    else:
        vals = rng.standard_normal(rows.size)
    zero = rng.random(rows.size) < zero_frac
    vals[zero] = 0.0
    lens = mask.sum(axis=1)
    row_ptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    return CSR(nrows, ncols, row_ptr.astype(np.int32), cols.astype(np.int32), vals)


def identity_csr(n: int) -> CSR:
    return CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
               np.ones(n))


def permute_fine(A: CSR, P: CSR, perm: np.ndarray):
    """Symmetric permutation of the fine index: A' = Q A Q^T, P' = Q P (perm[new] = old)."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)

    def rows_perm(M: CSR, remap_cols):
        lens = M.row_lengths()[perm]
        rp = np.zeros(M.nrows + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        cols = []
        vals = []
        for new, old in enumerate(perm):
            s, e = M.row_ptr[old], M.row_ptr[old + 1]
            c = M.col_idx[s:e].astype(np.int64)
            v = M.val[s:e]
            if remap_cols:
                c = inv[c]
                o = np.argsort(c)
                c, v = c[o], v[o]
            cols.append(c)
            vals.append(v)
        cc = np.concatenate(cols) if cols else np.zeros(0, np.int64)
        vv = np.concatenate(vals) if vals else np.zeros(0)
        return CSR(M.nrows, M.ncols, rp.astype(np.int32), cc.astype(np.int32), vv)

    return rows_perm(A, True), rows_perm(P, False)
