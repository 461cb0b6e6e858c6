"""The row-partitioned product (Section 2, Eq. 1-3; Alg. 7-10) with every rank's
local product, packing and reduction in the CUDA library.

One GPU stands in for the ranks by stepping them in lockstep in one process:
each rank's kernels run to completion before the host moves its exchange
buffers, so no kernel of one rank ever waits on another's.  The assembled
owned rows of every rank must equal the oracle's full product: pattern
exactly, values within tau * (|P|^T|A||P|)(i,j), for the merged loop
(Alg. 9-10) and the remote-first loop (Alg. 7-8), after a re-product with
new values.  Also checks ptap_gather / ptap_scatter_add on their own.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08423_gb300 import partition as pt
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from paper_1905_08423_gb300 import sharded as sh
from parity import TAU, rounded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_gather_scatter_add(dtype):
    g = torch.Generator().manual_seed(3)
    src = torch.randn(1000, generator=g, dtype=torch.float64).to(dtype).cuda()
    idx = torch.randperm(1000, generator=g)[:700].to(torch.int32).cuda()
    out = ptap.gather(src, idx)
    assert torch.equal(out, src[idx.long()])
    dst = torch.randn(1200, generator=g, dtype=torch.float64).to(dtype).cuda()
    want = dst.clone()
    pos = torch.randperm(1200, generator=g)[:700].to(torch.int32).cuda()
    want[pos.long()] += src[idx.long()]
    ptap.scatter_add(dst, pos, src, idx)
    assert torch.equal(dst, want)
    want[pos.long()] += src[:700]
    ptap.scatter_add(dst, pos, src)
    assert torch.equal(dst, want)


@pytest.mark.parametrize("kind", ["model", "algebraic"])
@pytest.mark.parametrize("merged", [True, False])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ranks_in_lockstep(kind, merged, dtype):
    A, P = pb.model_problem(31) if kind == "model" else pb.algebraic_problem(20, seed=7)
    world = 3
    fb = pt.block_bounds(A.nrows, world)
    ops = sh.LibraryOps("cuda", dtype)
    gens, blocks = [], []
    for r in range(world):
        Ab, Pb = sh.block_rows(A, int(fb[r]), int(fb[r + 1])), sh.block_rows(P, int(fb[r]), int(fb[r + 1]))
        blocks.append((Ab, Pb))
        gens.append(sh.setup(ops, Ab, Pb, A.nrows, P.ncols, r, world, merged))
    plans = sh.run_lockstep(gens)
    for scale in (1.0, 0.75):
        vals = [(torch.as_tensor(Ab.val * scale).to(dtype).cuda(), torch.as_tensor(Pb.val).to(dtype).cuda())
                for Ab, Pb in blocks]
        outs = sh.run_lockstep([sh.numeric(ops, p, a, q) for p, (a, q) in zip(plans, vals)])
        torch.cuda.synchronize()
        for p in plans:
            for part in p.parts:
                part.plan.check()
        Ar, Pr = rounded(A.with_values(A.val * scale), dtype), rounded(P, dtype)
        full, bnd = oracle.ptap(Ar, Pr), oracle.ptap_bound(Ar, Pr)
        for p, c in zip(plans, outs):
            a, b = full.row_ptr[p.c0], full.row_ptr[p.c1]
            np.testing.assert_array_equal(p.own_rp, full.row_ptr[p.c0:p.c1 + 1] - a)
            np.testing.assert_array_equal(p.own_ci, full.col_idx[a:b])
            err = np.abs(c.cpu().numpy().astype(np.float64) - full.val[a:b])
            B = bnd.val[a:b]
            assert np.all(np.where(B > 0, err <= TAU[dtype] * B, err == 0)), (p.rank, scale)
