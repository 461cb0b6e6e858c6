"""A multigrid hierarchy whose Galerkin operators come from the all-at-once product.

The paper's application builds a twelve-level method with eleven triple
products C = P^T A P (Section 4.2.2, Tables 5-6), one per level, in the
setup phase of its preconditioner, and repeats that setup as the operator's
values change.  ``Hierarchy`` does the same on one GPU: per level it
aggregates the rows (ptap_aggregate), forms the smoothed prolongator P =
(I - omega D^-1 A_F) T, A_F the operator filtered by strength theta
(ptap_prolongator_*; filtering keeps the coarse operators sparse, as the rows
of Tables 5-6 are), and forms the next operator with
ptap_symbolic / ptap_numeric; the coarse operator is the next level's A.

``renumeric`` re-runs only the numeric phases -- every level's P values and
product -- for new fine-level values on the fixed hierarchy (the paper's
repeated setup; Section 4.1's one symbolic, many numeric), and can be
captured once in a CUDA graph.  ``stats`` reports each level's operator and
prolongator in the layout of Tables 5 and 6.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import ptap


@dataclass
class Level:
    A: ptap.Csr                 # this level's operator
    agg: torch.Tensor           # aggregate of every row
    prol: ptap.Prolongator      # pattern of P
    P: ptap.Csr                 # P with its values
    plan: ptap.Plan             # symbolic result of P^T A P
    C: torch.Tensor             # values of the next level's operator


class Hierarchy:
    """Levels from the fine operator A (ptap.Csr, square, diagonal stored) down to
    at most ``coarse_rows`` rows or ``max_levels`` operators."""

    def __init__(self, A: ptap.Csr, max_levels: int = 12, coarse_rows: int = 400, passes: int = 2,
                 rounds: int = 16, omega: float = 2.0 / 3.0, theta: float = 0.5, config=None):
        self.omega, self.theta, self.passes, self.rounds = omega, theta, passes, rounds
        self.levels: list[Level] = []
        self.coarse: ptap.Csr = A
        cur = A
        while len(self.levels) + 1 < max_levels and cur.nrows > coarse_rows:
            agg, n_agg = ptap.aggregate(cur, passes, rounds)
            if n_agg >= cur.nrows:       # no coarsening possible
                break
            prol = ptap.Prolongator(cur, agg, n_agg, theta)
            P = prol.csr(prol.numeric(cur, omega))
            plan = ptap.symbolic(cur, P, config)
            C = ptap.numeric(plan, cur, P)
            rp, ci = plan.pattern()
            self.levels.append(Level(cur, agg, prol, P, plan, C))
            cur = ptap.Csr(plan.m, plan.m, rp, ci, C)
        self.coarse = cur

    def renumeric(self, A_val: torch.Tensor | None = None, stream=None):
        """Numeric phases only: every level's P values and triple product, from the fine
        operator's current values (or ``A_val``, copied into them first)."""
        if not self.levels:
            return
        if A_val is not None:
            self.levels[0].A.val.copy_(A_val)
        for lv in self.levels:
            lv.prol.numeric(lv.A, self.omega, out=lv.P.val, stream=stream)
            ptap.numeric(lv.plan, lv.A, lv.P, out=lv.C, stream=stream)

    def check(self):
        for lv in self.levels:
            lv.prol.check()
            lv.plan.check()

    def stats(self) -> dict:
        """Rows, nonzeros and per-row column counts of every operator (Table 5) and
        prolongator (Table 6)."""
        def rows(M):
            lens = torch.diff(M.row_ptr.long())
            return {"rows": M.nrows, "cols": M.ncols, "nonzeros": int(M.nnz),
                    "cols_min": int(lens.min()) if lens.numel() else 0,
                    "cols_max": int(lens.max()) if lens.numel() else 0,
                    "cols_avg": round(float(lens.float().mean()), 1) if lens.numel() else 0.0}
        ops = [rows(lv.A) for lv in self.levels] + [rows(self.coarse)]
        prols = [rows(lv.P) for lv in self.levels]
        return {"operators": ops, "interpolations": prols, "levels": len(ops), "products": len(prols)}

    def destroy(self):
        for lv in self.levels:
            lv.plan.destroy()
            lv.prol.destroy()
        self.levels = []
