"""CPU checks of the bookkeeping bench.py reports against: algorithmic bytes
and FMAs of one product, and the oracle's all-cores timing run."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1905_08423_gb300 import problems as pb

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _brute_fma(A, P):
    """sum_I sum_k nnz P(k,:) + nnz P(I,:) * nnz (A P)(I,:), counted row by row."""
    AP = oracle.spgemm(A, P)
    total = 0
    for I in range(A.nrows):
        for e in range(A.row_ptr[I], A.row_ptr[I + 1]):
            k = A.col_idx[e]
            total += int(P.row_ptr[k + 1] - P.row_ptr[k])
        total += int(P.row_ptr[I + 1] - P.row_ptr[I]) * int(AP.row_ptr[I + 1] - AP.row_ptr[I])
    return total


def test_fma_counts_agree():
    A, P = pb.model_problem(9)
    want = _brute_fma(A, P)
    assert bench.alg_fma_model(A, P, 9) == want
    assert bench.alg_fma_general(A, P, "cpu") == want
    A2, P2 = pb.algebraic_problem(7, seed=3)
    assert bench.alg_fma_general(A2, P2, "cpu") == _brute_fma(A2, P2)


def test_alg_bytes_definition():
    # row pointers, indices and values of A and P; C's pattern read; C's values written
    n, nnz_a, m, nnz_p, nnz_c = 10, 30, 4, 12, 9
    for vb in (4, 8):
        want = 4 * (n + 1) + (4 + vb) * nnz_a + 4 * (n + 1) + (4 + vb) * nnz_p + 4 * (m + 1) + 4 * nnz_c \
            + vb * nnz_c
        assert bench.alg_bytes(n, nnz_a, m, nnz_p, nnz_c, vb) == want


def test_parallel_oracle_baseline_runs():
    A, P = pb.model_problem(11)
    C = oracle.ptap(A, P)
    out = bench.cpu_baseline_parallel(A, P, int(C.row_ptr[-1]))
    assert out["kind"] == "oracle" and out["cores"] >= 1 and out["value"] > 0
    assert np.isfinite(out["value"])
