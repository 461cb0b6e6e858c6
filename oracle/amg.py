"""Oracle for the levels of the multigrid hierarchy: aggregation and the
smoothed prolongator.

TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded Python in FP64, used
to check the CUDA library's ptap_aggregate and ptap_prolongator_*.  Only
``tests/`` may import it.  It shares no code with the CUDA path.

The paper's hierarchy (Section 4.2.2: twelve levels, eleven triple products,
Tables 5-6) takes its coarsening from a cited work; the reading implemented
on both sides is smoothed aggregation:

* ``aggregate`` -- repeated pairwise matching.  In a round every unmatched
  node picks the unmatched neighbour node with the largest key (strength,
  edge_hash(a, b), then the smaller node on a full tie), the strength of two
  nodes being the largest |A(i,j)| between their members; nodes that picked
  each other form a pair.  Rounds repeat until none pairs or ``rounds`` is
  reached; then up to ``rounds`` more rounds key the edges by the hash alone.
  A node still unmatched joins the pair with which it has the strongest edge
  (alone only without a paired neighbour).  A pass turns pairs (with what
  joined them) and lone nodes into the next pass's nodes, numbered by their
  smaller old node.
* ``prolongator`` -- P = (I - omega D^-1 A_F) T with T(i, agg(i)) = 1, A_F the
  strength-filtered A and D = diag(A), on the pattern of A_F T (structural:
  entries are kept when their value is 0).
* ``greedy_matching`` -- an independent formulation of one pass run to
  convergence: sequential greedy matching over the edges in decreasing key
  order (the two agree when every edge has its own key).
"""
from __future__ import annotations

import numpy as np

_M32 = 0xFFFFFFFF


def edge_hash(a: int, b: int) -> int:
    """32-bit mix of the unordered node pair (a, b): the tie-break of equal strengths."""
    lo, hi = min(a, b), max(a, b)
    h = ((lo * 0x9E3779B1) & _M32) ^ ((hi + 0x7F4A7C15 + ((lo << 6) & _M32) + (lo >> 2)) & _M32)
    h &= _M32
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & _M32
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & _M32
    return h ^ (h >> 16)


def _node_edges(A, node_of, members, a):
    """Strongest |A(i,j)| from node a to every other node b, over a's members i."""
    rp, ci, v = A.row_ptr, A.col_idx, A.val
    best = {}
    for i in members[a]:
        for e in range(int(rp[i]), int(rp[i + 1])):
            b = node_of[int(ci[e])]
            if b == a:
                continue
            w = abs(float(v[e]))
            if b not in best or w > best[b]:
                best[b] = w
    return best


def aggregate(A, passes: int = 2, rounds: int = 16):
    """(agg, n_agg): the aggregate of every row of the square matrix A."""
    n = A.nrows
    node_of = list(range(n))
    members = [[i] for i in range(n)]
    for _ in range(passes):
        nn = len(members)
        if nn <= 1:
            break
        edges = [_node_edges(A, node_of, members, a) for a in range(nn)]
        partner = [-1] * nn
        for phase in ("strength", "hash"):
            for _ in range(rounds):
                pick = [-1] * nn
                for a in range(nn):
                    if partner[a] >= 0:
                        continue
                    cand = [(w if phase == "strength" else 0.0, edge_hash(a, b), -b)
                            for b, w in edges[a].items() if partner[b] < 0]
                    if cand:
                        pick[a] = -max(cand)[2]
                matched = 0
                for a in range(nn):
                    b = pick[a]
                    if b >= 0 and pick[b] == a:
                        partner[a] = b
                        matched += a < b
                if matched == 0:
                    break
        # an unmatched node joins the pair it has the strongest edge with
        att = [-1] * nn
        for a in range(nn):
            if partner[a] >= 0:
                continue
            cand = [(w, edge_hash(a, b), -b) for b, w in edges[a].items() if partner[b] >= 0]
            if cand:
                b = -max(cand)[2]
                att[a] = min(b, partner[b])
        leader = [min(a, partner[a]) if partner[a] >= 0 else (att[a] if att[a] >= 0 else a)
                  for a in range(nn)]
        leaders = [a for a in range(nn) if leader[a] == a]
        new_id = {a: k for k, a in enumerate(leaders)}
        new_members = [[] for _ in leaders]
        for a in range(nn):
            new_members[new_id[leader[a]]].extend(members[a])
        for k, mem in enumerate(new_members):
            for i in mem:
                node_of[i] = k
        members = new_members
        assert len(new_id) == len(members)
    return np.asarray(node_of, dtype=np.int32), len(members)


def greedy_matching(A):
    """Pairs of one pass on the rows of A by sequential greedy matching: edges in
    decreasing (|A(i,j)|, edge_hash) order, an edge taken when both ends are free."""
    n = A.nrows
    keys = {}
    for i in range(n):
        for e in range(int(A.row_ptr[i]), int(A.row_ptr[i + 1])):
            j = int(A.col_idx[e])
            if j == i:
                continue
            a, b = min(i, j), max(i, j)
            w = abs(float(A.val[e]))
            keys[(a, b)] = max(keys.get((a, b), -1.0), w)
    order = sorted(keys, key=lambda ab: (keys[ab], edge_hash(*ab), -ab[0], -ab[1]), reverse=True)
    partner = [-1] * n
    for a, b in order:
        if partner[a] < 0 and partner[b] < 0:
            partner[a], partner[b] = b, a
    return partner


def prolongator(A, agg, n_agg: int, omega: float = 2.0 / 3.0, theta: float = 0.0, S=None):
    """P = (I - omega D^-1 A_F) T as (row_ptr, col_idx, val) on the pattern of A_F T.

    A_F keeps the diagonal and the off-diagonal entries with |A(i,j)| >=
    theta * max_{k != i} |A(i,k)|; D = diag(A).  Structural: entries are
    kept when their value is zero.  S (A's pattern, other values) decides the strong entries
    instead of A when given: a hierarchy settles them once, at setup.
    """
    S = A if S is None else S
    n = A.nrows
    rp_out, ci_out, val_out = [0], [], []
    for i in range(n):
        lo, hi = int(A.row_ptr[i]), int(A.row_ptr[i + 1])
        off = [e for e in range(lo, hi) if int(A.col_idx[e]) != i]
        mx = max((abs(float(S.val[e])) for e in off), default=0.0)
        strong = [e for e in off if abs(float(S.val[e])) >= theta * mx]
        d = [float(A.val[e]) for e in range(lo, hi) if int(A.col_idx[e]) == i][0]
        cols = sorted({int(agg[int(A.col_idx[e])]) for e in strong} | {int(agg[i])})
        row = {c: 0.0 for c in cols}
        row[int(agg[i])] = 1.0 - omega          # the diagonal term: omega * A(i,i) / A(i,i)
        for e in strong:
            row[int(agg[int(A.col_idx[e])])] -= omega / d * float(A.val[e])
        ci_out.extend(cols)
        val_out.extend(row[c] for c in cols)
        rp_out.append(len(ci_out))
    return (np.asarray(rp_out, dtype=np.int64), np.asarray(ci_out, dtype=np.int64),
            np.asarray(val_out, dtype=np.float64))
