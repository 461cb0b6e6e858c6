// Backward of C = P^T A P (not in the paper; follows from Eq. 7 by the chain
// rule).  With G = dL/dC stored on C's pattern,
//
//   dL/dA = P G P^T              restricted to pat(A)
//   dL/dP = A P G^T + A^T P G    restricted to pat(P)
//
// computed row by row without forming any product matrix:
//
//   dA(I,J)            = sum_{i in P(I,:)} P(I,i) <G(i,:), P(J,:)>
//   (A P G^T)(I,j)     = sum_{k in A(I,:)} A(I,k) <P(k,:), G(j,:)>     j in P(I,:)
//   (A^T P G)(J,j)    += A(I,J) sum_{i in P(I,:)} P(I,i) G(i,j)        J in A(I,:), j in P(J,:)
//
// Each <x, y> is a merge of two rows with sorted columns.  The first two are
// owned by fine row I and stored directly; the third scatters into other rows
// and is added with atomics in a second kernel, after the first has written
// dP.
#include <algorithm>

#include "owner.cuh"

namespace ptap {

template <typename V>
__device__ __forceinline__ V sorted_dot(const int32_t* __restrict__ ca, const V* __restrict__ va,
                                        int32_t a0, int32_t a1, const int32_t* __restrict__ cb,
                                        const V* __restrict__ vb, int32_t b0, int32_t b1) {
  V s = V(0);
  while (a0 < a1 && b0 < b1) {
    const int32_t x = ca[a0], y = cb[b0];
    if (x == y) {
      s += va[a0] * vb[b0];
      ++a0;
      ++b0;
    } else if (x < y) {
      ++a0;
    } else {
      ++b0;
    }
  }
  return s;
}

template <typename V>
struct BwdArgs {
  CsrV<V> A, P;
  const int32_t* c_rp;
  const int32_t* c_ci;
  const V* G;
  V* dA;
  V* dP;
};

// One thread per (fine row, entry of A(I,:)) for dA, and per (fine row,
// entry of P(I,:)) for the A P G^T part of dP.  Entries are found from the
// flat index by a binary search on the row pointer.
__device__ __forceinline__ int32_t row_of(const int32_t* __restrict__ rp, int32_t nrows, int64_t e) {
  int32_t lo = 0, hi = nrows - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (rp[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename V>
__global__ void k_bwd_dA(BwdArgs<V> a, int64_t nnz_a) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_a;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t I = row_of(a.A.rp, a.A.nrows, e);
    const int32_t J = a.A.ci[e];
    V s = V(0);
    const int32_t pj0 = a.P.rp[J], pj1 = a.P.rp[J + 1];
    for (int32_t q = a.P.rp[I]; q < a.P.rp[I + 1]; ++q) {
      const int32_t i = a.P.ci[q];
      s += a.P.val[q] * sorted_dot(a.c_ci, a.G, a.c_rp[i], a.c_rp[i + 1], a.P.ci, a.P.val, pj0, pj1);
    }
    a.dA[e] = s;
  }
}

template <typename V>
__global__ void k_bwd_dP_own(BwdArgs<V> a, int64_t nnz_p) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_p;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t I = row_of(a.P.rp, a.P.nrows, e);
    const int32_t j = a.P.ci[e];
    const int32_t g0 = a.c_rp[j], g1 = a.c_rp[j + 1];
    V s = V(0);
    for (int32_t x = a.A.rp[I]; x < a.A.rp[I + 1]; ++x) {
      const int32_t k = a.A.ci[x];
      s += a.A.val[x] * sorted_dot(a.P.ci, a.P.val, a.P.rp[k], a.P.rp[k + 1], a.c_ci, a.G, g0, g1);
    }
    a.dP[e] = s;
  }
}

// (A^T P G)(J, j) += A(I,J) (P G)(I, j): one thread per entry (I,J) of A.
template <typename V>
__global__ void k_bwd_dP_scatter(BwdArgs<V> a, int64_t nnz_a) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_a;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t I = row_of(a.A.rp, a.A.nrows, e);
    const int32_t J = a.A.ci[e];
    const V aIJ = a.A.val[e];
    const int32_t q0 = a.P.rp[I], q1 = a.P.rp[I + 1];
    if (q0 == q1) continue;
    for (int32_t b = a.P.rp[J]; b < a.P.rp[J + 1]; ++b) {
      const int32_t j = a.P.ci[b];
      V pg = V(0);
      for (int32_t q = q0; q < q1; ++q) {
        const int32_t i = a.P.ci[q];
        const int32_t pos = find_col(a.c_ci, a.c_rp[i], a.c_rp[i + 1], j);
        if (pos >= 0) pg += a.P.val[q] * a.G[pos];
      }
      if (pg != V(0)) atomicAdd(&a.dP[b], aIJ * pg);
    }
  }
}

template <typename V>
static int backward_t(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, const void* G, void* dA,
                      void* dP, cudaStream_t s) {
  BwdArgs<V> a;
  a.A = CsrV<V>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const V*)A->val};
  a.P = CsrV<V>{P->nrows, P->ncols, P->row_ptr, P->col_idx, (const V*)P->val};
  a.c_rp = p->c_rp;
  a.c_ci = p->c_ci;
  a.G = (const V*)G;
  a.dA = (V*)dA;
  a.dP = (V*)dP;
  const int grid = num_sms() * 16, threads = 256;
  if (dA && p->nnz_a > 0) {
    k_bwd_dA<V><<<(unsigned)std::min<int64_t>(grid, ceil_div(p->nnz_a, threads)), threads, 0, s>>>(
        a, p->nnz_a);
    PTAP_LAUNCHED();
  }
  if (dP && p->nnz_p > 0) {
    k_bwd_dP_own<V><<<(unsigned)std::min<int64_t>(grid, ceil_div(p->nnz_p, threads)), threads, 0, s>>>(
        a, p->nnz_p);
    PTAP_LAUNCHED();
    if (p->nnz_a > 0) {
      k_bwd_dP_scatter<V><<<(unsigned)std::min<int64_t>(grid, ceil_div(p->nnz_a, threads)), threads, 0,
                            s>>>(a, p->nnz_a);
      PTAP_LAUNCHED();
    }
  }
  return PTAP_OK;
}

int check_numeric_inputs(const ptap_plan* p, const ptap_csr* A, const ptap_csr* P);

}  // namespace ptap

extern "C" int ptap_backward(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, const void* G,
                             void* dA, void* dP, void* stream) {
  ptap::Range range("ptap_backward");
  if (!p) return PTAP_ERR_INVALID;
  PTAP_TRY(ptap::check_numeric_inputs(p, A, P));
  if (p->nnz_c > 0 && !G) return PTAP_ERR_INVALID;
  if (p->n == 0) return PTAP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->dtype == PTAP_F64) return ptap::backward_t<double>(p, A, P, G, dA, dP, s);
  return ptap::backward_t<float>(p, A, P, G, dA, dP, s);
}
