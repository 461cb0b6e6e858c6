// GPU two-step comparator (Section 3, Eq. 6; Alg. 5 symbolic, Alg. 6 numeric):
//
//   C~ = A P     (row-wise product, Alg. 3-4)
//   P^T          (explicit transpose, pattern + values)
//   C  = P^T C~  (row-wise product again)
//
// The plan holds C~ (pattern and values) and P^T (pattern, the permutation
// into P, and values): exactly the auxiliary matrices whose memory the paper's
// all-at-once algorithms avoid.  The numeric phase is the same row-wise hash
// kernel applied twice, plus a gather for P^T's values.
#include <algorithm>
#include <new>

#include "owner.cuh"

namespace ptap {

int symbolic_prologue(const ptap_csr* A, const ptap_csr* P, const ptap_config* cfg,
                      const ptap_allocator* alloc, void* stream, ptap_plan** out, int kind);
int union_pattern_ab(Tracker& mem, const CsrI& A, const CsrI& B, const Config& cfg, int32_t* rp,
                     int32_t** ci, int64_t* nnz, int32_t* status, int* spilled, cudaStream_t s);

struct TwoStepData {
  int32_t* ap_rp = nullptr;
  int32_t* ap_ci = nullptr;
  void* ap_val = nullptr;
  int64_t nnz_ap = 0;
  int32_t* pt_rp = nullptr;
  int32_t* pt_ci = nullptr;
  int32_t* pt_perm = nullptr;
  void* pt_val = nullptr;
};

// Row-wise numeric product C = A B into a known sorted pattern: one group of
// G lanes per output row, a hash map per group; overflowing rows add their
// products straight into C with atomics (only that group touches the row).
template <typename V, int G>
__global__ void __launch_bounds__(256) k_rowwise_numeric(CsrV<V> A, CsrV<V> B, const int32_t* c_rp,
                                                        const int32_t* c_ci, V* c_val, int slots_log2,
                                                        int32_t* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t gflag[256 / 4];
  const int slots = 1 << slots_log2;
  const int group = threadIdx.x / G, glane = threadIdx.x % G, ngroups = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  V* hv = (V*)smraw + group * slots;
  int32_t* hk = (int32_t*)((V*)smraw + ngroups * slots) + group * slots;
  for (int64_t rg = (int64_t)blockIdx.x * ngroups + group; rg < A.nrows;
       rg += (int64_t)gridDim.x * ngroups) {
    const int32_t r = (int32_t)rg;
    const int32_t c0 = c_rp[r], c1 = c_rp[r + 1];
    if (c0 == c1) continue;
    for (int s = glane; s < slots; s += G) {
      hk[s] = kEmpty;
      hv[s] = V(0);
    }
    if (glane == 0) gflag[group] = 0;
    __syncwarp(gmask);
    const int32_t a0 = A.rp[r], a1 = A.rp[r + 1];
    for (int32_t x = a0 + glane; x < a1; x += G) {
      const int32_t k = A.ci[x];
      const V av = A.val[x];
      for (int32_t b = B.rp[k]; b < B.rp[k + 1]; ++b) {
        if (((volatile int32_t*)gflag)[group]) break;
        const int sl = map_slot(hk, slots_log2, B.ci[b]);
        if (sl < 0) {
          gflag[group] = 1;
          break;
        }
        atomicAdd(&hv[sl], av * B.val[b]);
      }
    }
    __syncwarp(gmask);
    if (!((volatile int32_t*)gflag)[group]) {
      for (int s = glane; s < slots; s += G) {
        const int32_t j = hk[s];
        if (j == kEmpty) continue;
        const int32_t pos = find_col(c_ci, c0, c1, j);
        if (pos >= 0) c_val[pos] = hv[s];
        else atomicExch(status, PTAP_ERR_PATTERN);
      }
    } else {
      for (int32_t e = c0 + glane; e < c1; e += G) c_val[e] = V(0);
      __syncwarp(gmask);
      for (int32_t x = a0 + glane; x < a1; x += G) {
        const int32_t k = A.ci[x];
        const V av = A.val[x];
        for (int32_t b = B.rp[k]; b < B.rp[k + 1]; ++b) {
          const int32_t pos = find_col(c_ci, c0, c1, B.ci[b]);
          if (pos >= 0) atomicAdd(&c_val[pos], av * B.val[b]);
          else atomicExch(status, PTAP_ERR_PATTERN);
        }
      }
    }
    __syncwarp(gmask);
  }
}

template <typename V>
__global__ void k_gather_vals(const V* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                              V* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[perm[t]];
}

template <typename V, int G>
static int launch_rowwise_g(const CsrV<V>& A, const CsrV<V>& B, const int32_t* rp, const int32_t* ci,
                            V* val, const Config& c, int32_t* status, cudaStream_t s) {
  const int threads = c.block_threads;
  const int slots_log2 = c.force_spill ? 2 : ilog2_ceil((uint32_t)std::max(4, c.ap_slots));
  const size_t smem = (size_t)(threads / G) * (1 << slots_log2) * (sizeof(V) + sizeof(int32_t));
  PTAP_TRY(grow_smem_limit((const void*)k_rowwise_numeric<V, G>, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rowwise_numeric<V, G>, threads, smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  if (A.nrows == 0) return PTAP_OK;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(ceil_div(A.nrows, threads / G), (int64_t)num_sms() * per_sm));
  k_rowwise_numeric<V, G><<<grid, threads, smem, s>>>(A, B, rp, ci, val, slots_log2, status);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

template <typename V>
static int launch_rowwise(const CsrV<V>& A, const CsrV<V>& B, const int32_t* rp, const int32_t* ci,
                          V* val, const Config& c, int32_t* status, cudaStream_t s) {
  switch (c.group_lanes) {
    case 4: return launch_rowwise_g<V, 4>(A, B, rp, ci, val, c, status, s);
    case 8: return launch_rowwise_g<V, 8>(A, B, rp, ci, val, c, status, s);
    case 16: return launch_rowwise_g<V, 16>(A, B, rp, ci, val, c, status, s);
    case 32: return launch_rowwise_g<V, 32>(A, B, rp, ci, val, c, status, s);
  }
  return PTAP_ERR_INVALID;
}

template <typename V>
static int two_step_numeric_t(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C,
                              cudaStream_t s) {
  TwoStepData* t = p->two;
  // Alg. 6 line 2: C~ = A P
  CsrV<V> Av{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const V*)A->val};
  CsrV<V> Pv{P->nrows, P->ncols, P->row_ptr, P->col_idx, (const V*)P->val};
  PTAP_TRY(launch_rowwise<V>(Av, Pv, t->ap_rp, t->ap_ci, (V*)t->ap_val, p->cfg, p->status, s));
  // Alg. 6 line 3: numeric transpose of P
  if (p->nnz_p > 0) {
    k_gather_vals<V><<<num_sms() * 8, 256, 0, s>>>((const V*)P->val, t->pt_perm, p->nnz_p,
                                                   (V*)t->pt_val);
    PTAP_LAUNCHED();
  }
  // Alg. 6 lines 4-8 (one process): C = P^T C~
  CsrV<V> Ptv{p->m, p->n, t->pt_rp, t->pt_ci, (const V*)t->pt_val};
  CsrV<V> APv{p->n, p->m, t->ap_rp, t->ap_ci, (const V*)t->ap_val};
  return launch_rowwise<V>(Ptv, APv, p->c_rp, p->c_ci, (V*)C, p->cfg, p->status, s);
}

int two_step_numeric(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  if (p->dtype == PTAP_F64) return two_step_numeric_t<double>(p, A, P, C, s);
  return two_step_numeric_t<float>(p, A, P, C, s);
}

void two_step_free(ptap_plan* p) {
  delete p->two;
  p->two = nullptr;
}

static int two_step_body(ptap_plan* p, const ptap_csr* A, const ptap_csr* P) {
  cudaStream_t s = p->stream;
  p->two = new (std::nothrow) TwoStepData();
  if (!p->two) return PTAP_ERR_OOM;
  TwoStepData* t = p->two;
  const size_t vb = p->dtype == PTAP_F64 ? 8 : 4;
  CsrI Ai{A->nrows, A->ncols, A->row_ptr, A->col_idx};
  CsrI Pi{P->nrows, P->ncols, P->row_ptr, P->col_idx};
  // Alg. 5 line 2: pattern of C~ = A P
  PTAP_TRY(p->mem.get_n(&t->ap_rp, (int64_t)p->n + 1));
  int spilled = 0;
  PTAP_TRY(union_pattern_ab(p->mem, Ai, Pi, p->cfg, t->ap_rp, &t->ap_ci, &t->nnz_ap, p->status,
                            &spilled, s));
  // Alg. 5 line 3: explicit symbolic transpose of P
  PTAP_TRY(p->mem.get_n(&t->pt_rp, (int64_t)p->m + 1));
  PTAP_TRY(p->mem.get_n(&t->pt_ci, p->nnz_p));
  PTAP_TRY(p->mem.get_n(&t->pt_perm, p->nnz_p));
  PTAP_TRY(transpose_pattern(p->mem, Pi, t->pt_rp, t->pt_ci, t->pt_perm, s));
  // Alg. 5 lines 4-8: pattern of C = P^T C~
  PTAP_TRY(p->mem.get_n(&p->c_rp, (int64_t)p->m + 1));
  CsrI Pti{p->m, p->n, t->pt_rp, t->pt_ci};
  CsrI APi{p->n, p->m, t->ap_rp, t->ap_ci};
  int spilled2 = 0;
  PTAP_TRY(union_pattern_ab(p->mem, Pti, APi, p->cfg, p->c_rp, &p->c_ci, &p->nnz_c, p->status,
                            &spilled2, s));
  p->spill_rows = spilled + spilled2;
  // value storage of the auxiliary matrices
  PTAP_TRY(p->mem.get(&t->ap_val, (size_t)t->nnz_ap * vb));
  PTAP_TRY(p->mem.get(&t->pt_val, (size_t)p->nnz_p * vb));
  PTAP_CUDA(cudaStreamSynchronize(s));
  int32_t st = 0;
  PTAP_CUDA(cudaMemcpy(&st, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (st) return st;
  p->symbolic_peak = p->mem.peak;
  return PTAP_OK;
}

}  // namespace ptap

extern "C" int ptap_two_step_symbolic(const ptap_csr* A, const ptap_csr* P, const ptap_config* cfg,
                                      const ptap_allocator* alloc, void* stream, ptap_plan** out) {
  ptap::Range range("ptap_two_step_symbolic");
  ptap_plan* p = nullptr;
  PTAP_TRY(ptap::symbolic_prologue(A, P, cfg, alloc, stream, &p, 1));
  int rc = ptap::two_step_body(p, A, P);
  if (rc != PTAP_OK) {
    cudaStreamSynchronize(p->stream);
    p->mem.release_all();
    ptap::two_step_free(p);
    delete p;
    return rc;
  }
  *out = p;
  return PTAP_OK;
}
