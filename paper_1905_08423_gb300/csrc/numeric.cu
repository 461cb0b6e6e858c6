// Numeric phase of the all-at-once triple product (Section 3, Eq. 9, Alg. 8).
//
//   C = sum_I  P(I,:)^T  x  (A P)(I,:)
//
// For each fine row I the row R = (A P)(I,:) is formed in a hash map
// (Alg. 3: R(j) += A(I,k) P(k,j)), and the outer product P(I,:)^T x R is added
// straight into the preallocated C; neither A P nor P^T is stored.
//
// Two schemes:
//
// * OWNER (default).  The coarse rows are cut into chunks whose C entries fit
//   in shared memory.  One CTA owns a chunk: it loads the chunk's sorted C
//   column indices, zeroes an on-chip accumulator, visits every fine row I
//   whose P(I,:) reaches into the chunk (the plan's per-chunk list), forms R
//   once per visit, adds P(I,i) R for the i inside the chunk, and finally
//   writes the chunk's values to C exactly once.  No memset of C, no global
//   atomics; the price is that a fine row bordering two chunks forms its R
//   row in both.
// * ATOMIC.  The paper's loop taken literally: every fine row forms R once
//   and scatters into C with global atomics (C zeroed first).
//
// Rows of A P that overflow a group's hash map fall back to adding the
// individual products A(I,k) P(k,j) P(I,i) without merging them first, which
// needs no table at all.
#include <algorithm>

#include "owner.cuh"

namespace ptap {

// ---------------------------------------------------------------------------
// OWNER scheme
// ---------------------------------------------------------------------------
template <typename V, int G>
__global__ void __launch_bounds__(256) k_numeric_owner(NumArgs<V> a, int slots_log2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t gflag[256 / 4];
  OwnerSmem<V> sm(smraw, a.CH, a.max_rows, blockDim.x / G, 1 << slots_log2);
  for (int32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x)
    owner_chunk<V, G>(a, c, sm, gflag, slots_log2);
}

// ---------------------------------------------------------------------------
// ATOMIC scheme (Alg. 8 literally; C must be zeroed first)
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ void global_add(const NumArgs<V>& a, int32_t i, int32_t j, V wv) {
  const int32_t pos = find_col(a.c_ci, a.c_rp[i], a.c_rp[i + 1], j);
  if (pos >= 0) atomicAdd(&a.c_val[pos], wv);
  else atomicExch(a.status, PTAP_ERR_PATTERN);
}

template <typename V, int G>
__global__ void __launch_bounds__(256) k_numeric_atomic(NumArgs<V> a, int slots_log2) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t gflag[256 / 4];
  const int slots = 1 << slots_log2;
  const int group = threadIdx.x / G, glane = threadIdx.x % G, ngroups = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  V* hv = (V*)smraw + group * slots;
  int32_t* hk = (int32_t*)((V*)smraw + ngroups * slots) + group * slots;
  const int32_t n = a.A.nrows;
  for (int64_t Ig = (int64_t)blockIdx.x * ngroups + group; Ig < n; Ig += (int64_t)gridDim.x * ngroups) {
    const int32_t I = (int32_t)Ig;
    const int32_t p0 = a.P.rp[I], p1 = a.P.rp[I + 1];
    if (p0 == p1) continue;  // empty P(I,:) contributes nothing (Alg. 7-8)
    for (int s = glane; s < slots; s += G) {
      hk[s] = kEmpty;
      hv[s] = V(0);
    }
    if (glane == 0) gflag[group] = 0;
    __syncwarp(gmask);
    const int32_t a0 = a.A.rp[I], a1 = a.A.rp[I + 1];
    for (int32_t x = a0 + glane; x < a1; x += G) {
      const int32_t k = a.A.ci[x];
      const V av = a.A.val[x];
      for (int32_t b = a.P.rp[k]; b < a.P.rp[k + 1]; ++b) {
        if (((volatile int32_t*)gflag)[group]) break;
        const int sl = map_slot(hk, slots_log2, a.P.ci[b]);
        if (sl < 0) {
          gflag[group] = 1;
          break;
        }
        atomicAdd(&hv[sl], av * a.P.val[b]);
      }
    }
    __syncwarp(gmask);
    if (!((volatile int32_t*)gflag)[group]) {
      for (int s = glane; s < slots; s += G) {
        const int32_t j = hk[s];
        if (j == kEmpty) continue;
        const V v = hv[s];
        for (int32_t e = p0; e < p1; ++e) global_add(a, a.P.ci[e], j, a.P.val[e] * v);
      }
    } else {
      for (int32_t x = a0 + glane; x < a1; x += G) {
        const int32_t k = a.A.ci[x];
        const V av = a.A.val[x];
        for (int32_t b = a.P.rp[k]; b < a.P.rp[k + 1]; ++b) {
          const V t = av * a.P.val[b];
          for (int32_t e = p0; e < p1; ++e) global_add(a, a.P.ci[e], a.P.ci[b], a.P.val[e] * t);
        }
      }
    }
    __syncwarp(gmask);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename V>
static NumArgs<V> make_args(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C) {
  NumArgs<V> a;
  a.A = CsrV<V>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const V*)A->val};
  a.P = CsrV<V>{P->nrows, P->ncols, P->row_ptr, P->col_idx, (const V*)P->val};
  a.c_rp = p->c_rp;
  a.c_ci = p->c_ci;
  a.c_val = (V*)C;
  a.chunk_row = p->chunk_row;
  a.chunk_fptr = p->chunk_fptr;
  a.chunk_frows = p->chunk_frows;
  a.nchunks = p->nchunks;
  a.CH = p->cfg.chunk_entries;
  a.max_rows = std::max(p->max_chunk_rows, 1);
  a.status = p->status;
  return a;
}

static int slots_log2_of(const Config& c) {
  int s = c.force_spill ? 2 : ilog2_ceil((uint32_t)std::max(4, c.ap_slots));
  return s;
}

template <typename V>
size_t owner_smem_bytes(const Config& c, int max_rows, int threads) {
  const int slots = 1 << slots_log2_of(c);
  const int groups = threads / c.group_lanes;
  size_t b = (size_t)c.chunk_entries * sizeof(V) + (size_t)groups * slots * sizeof(V);
  b += ((size_t)c.chunk_entries + max_rows + 1 + (size_t)groups * slots) * sizeof(int32_t);
  return (b + 15) & ~size_t(15);
}

// Kernel attributes and occupancy are settled once, when the plan is built,
// so that the numeric launch itself is a single kernel launch (and can be
// captured in a CUDA graph).
template <typename V, int G>
static int prepare_owner_g(ptap_plan* p) {
  const Config& c = p->cfg;
  const size_t smem = owner_smem_bytes<V>(c, std::max(p->max_chunk_rows, 1), c.block_threads);
  PTAP_TRY(grow_smem_limit((const void*)k_numeric_owner<V, G>, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_numeric_owner<V, G>,
                                                          c.block_threads, smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  p->num_smem = smem;
  p->num_per_sm = per_sm;
  return PTAP_OK;
}

template <typename V, int G>
static int launch_owner_g(ptap_plan* p, const NumArgs<V>& a, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(a.nchunks, (int64_t)num_sms() * p->num_per_sm);
  if (grid <= 0) return PTAP_OK;
  k_numeric_owner<V, G><<<grid, p->cfg.block_threads, p->num_smem, s>>>(a, slots_log2_of(p->cfg));
  PTAP_LAUNCHED();
  return PTAP_OK;
}

template <typename V, int G>
static int prepare_atomic_g(ptap_plan* p) {
  const Config& c = p->cfg;
  const int slots = 1 << slots_log2_of(c);
  const size_t smem = (size_t)(c.block_threads / G) * slots * (sizeof(V) + sizeof(int32_t));
  PTAP_TRY(grow_smem_limit((const void*)k_numeric_atomic<V, G>, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_numeric_atomic<V, G>,
                                                          c.block_threads, smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  p->num_smem = smem;
  p->num_per_sm = per_sm;
  return PTAP_OK;
}

template <typename V, int G>
static int launch_atomic_g(ptap_plan* p, const NumArgs<V>& a, cudaStream_t s) {
  const int threads = p->cfg.block_threads;
  const int64_t groups_needed = ceil_div(a.A.nrows, threads / G);
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(groups_needed, (int64_t)num_sms() * p->num_per_sm));
  k_numeric_atomic<V, G><<<grid, threads, p->num_smem, s>>>(a, slots_log2_of(p->cfg));
  PTAP_LAUNCHED();
  return PTAP_OK;
}

// Calls F<V, G>() for the plan's dtype and group width.
#define PTAP_DISPATCH_VG(p, CALL)                                   \
  do {                                                              \
    const int _g = (p)->cfg.group_lanes;                            \
    if ((p)->dtype == PTAP_F64) {                                   \
      using V = double;                                             \
      if (_g == 4) { constexpr int G = 4; return CALL; }            \
      if (_g == 8) { constexpr int G = 8; return CALL; }            \
      if (_g == 16) { constexpr int G = 16; return CALL; }          \
      if (_g == 32) { constexpr int G = 32; return CALL; }          \
    } else {                                                        \
      using V = float;                                              \
      if (_g == 4) { constexpr int G = 4; return CALL; }            \
      if (_g == 8) { constexpr int G = 8; return CALL; }            \
      if (_g == 16) { constexpr int G = 16; return CALL; }          \
      if (_g == 32) { constexpr int G = 32; return CALL; }          \
    }                                                               \
    return PTAP_ERR_INVALID;                                        \
  } while (0)

int prepare_fast(ptap_plan* p);
int numeric_fast(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s);
int prepare_sorted(ptap_plan* p);  // sorted.cu
template <typename V>
int launch_sorted_t(ptap_plan* p, const NumArgs<V>& a, cudaStream_t s);

// The general owner-mode kernel: sort-based unless the hash groups were asked
// for, or tiny tables are forced (which exercises the hash path's spills).
static bool use_sorted(const ptap_plan* p) { return p->cfg.general_kernel == 0 && !p->cfg.force_spill; }

int prepare_numeric(ptap_plan* p) {
  if (p->cfg.mode == PTAP_MODE_ATOMIC) PTAP_DISPATCH_VG(p, (prepare_atomic_g<V, G>(p)));
  if (p->fast) return prepare_fast(p);
  if (use_sorted(p)) return prepare_sorted(p);
  PTAP_DISPATCH_VG(p, (prepare_owner_g<V, G>(p)));
}

int numeric_owner(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  if (p->nchunks == 0) return PTAP_OK;
  if (p->fast) return numeric_fast(p, A, P, C, s);
  if (use_sorted(p))
    return p->dtype == PTAP_F64 ? launch_sorted_t<double>(p, make_args<double>(p, A, P, C), s)
                                : launch_sorted_t<float>(p, make_args<float>(p, A, P, C), s);
  PTAP_DISPATCH_VG(p, (launch_owner_g<V, G>(p, make_args<V>(p, A, P, C), s)));
}

int numeric_atomic(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  const size_t vb = p->dtype == PTAP_F64 ? 8 : 4;
  if (p->nnz_c > 0) PTAP_CUDA(cudaMemsetAsync(C, 0, (size_t)p->nnz_c * vb, s));
  if (p->n == 0) return PTAP_OK;
  PTAP_DISPATCH_VG(p, (launch_atomic_g<V, G>(p, make_args<V>(p, A, P, C), s)));
}

// Owner-mode shared memory per CTA (exported for the batched kernel's sizing).
size_t owner_smem_for(int dtype, const Config& c, int max_rows) {
  return dtype == PTAP_F64 ? owner_smem_bytes<double>(c, max_rows, c.block_threads)
                           : owner_smem_bytes<float>(c, max_rows, c.block_threads);
}

int check_numeric_inputs(const ptap_plan* p, const ptap_csr* A, const ptap_csr* P) {
  PTAP_TRY(check_csr_host(A, true));
  PTAP_TRY(check_csr_host(P, true));
  if (A->dtype != p->dtype || P->dtype != p->dtype) return PTAP_ERR_INVALID;
  if (A->nrows != p->n || A->ncols != p->n || P->nrows != p->n || P->ncols != p->m ||
      A->nnz != p->nnz_a || P->nnz != p->nnz_p)
    return PTAP_ERR_PATTERN;
  return PTAP_OK;
}

}  // namespace ptap

extern "C" int ptap_numeric(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C_val,
                            void* stream) {
  ptap::Range range("ptap_numeric");
  if (!p) return PTAP_ERR_INVALID;
  PTAP_TRY(ptap::check_numeric_inputs(p, A, P));
  if (p->nnz_c > 0 && !C_val) return PTAP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (p->kind == 1) return ptap::two_step_numeric(p, A, P, C_val, s);
  if (p->cfg.mode == PTAP_MODE_ATOMIC) return ptap::numeric_atomic(p, A, P, C_val, s);
  return ptap::numeric_owner(p, A, P, C_val, s);
}
