// Symbolic phase of the all-at-once triple product (Section 3, Alg. 7).
//
// The paper accumulates the pattern of C with one hash set per C row, fed by
// outer products P(I,:) x R where R is the pattern of one row of A P (Alg. 1).
// On one GPU the same set is built row-owned ("pull"): coarse row i of C is
//
//     pattern(C(i,:)) = U_{I : P(I,i) in pat(P)}  U_{k in A(I,:)}  pattern(P(k,:))
//
// which needs the pattern of P's columns (a transient transpose, freed before
// the numeric phase) and no auxiliary A P.  Each row's union lives in an
// open-addressing table: a warp-private table in shared memory first, a
// CTA-wide one for rows that overflow it, and a global-memory table from a
// pooled arena for the rest (the heavy-row spill).  Counts are scanned into
// row_ptr ("preallocate", Alg. 7), then a second pass writes each row's keys
// in ascending order.  No floating point is touched.
#include <algorithm>
#include <new>

#include "common.cuh"

namespace ptap {

// ---------------------------------------------------------------------------
// expansion of one output row into candidate column keys
// ---------------------------------------------------------------------------
// Rows of P^T A P: i -> I in P^T(i,:) -> k in A(I,:) -> j in P(k,:).
struct Expand3 {
  CsrI Pt, A, P;
  template <class F>
  __device__ void run(int32_t row, int lane, int nl, const volatile int32_t* stop, F&& f) const {
    const int32_t e1 = Pt.rp[row + 1];
    for (int32_t e = Pt.rp[row] + lane; e < e1; e += nl) {
      const int32_t I = Pt.ci[e];
      const int32_t a1 = A.rp[I + 1];
      for (int32_t a = A.rp[I]; a < a1; ++a) {
        const int32_t k = A.ci[a];
        const int32_t b1 = P.rp[k + 1];
        for (int32_t b = P.rp[k]; b < b1; ++b) {
          if (*stop) return;
          f(P.ci[b]);
        }
      }
    }
  }
  __device__ int64_t bound(int32_t row) const {
    int64_t s = 0;
    for (int32_t e = Pt.rp[row]; e < Pt.rp[row + 1]; ++e) {
      const int32_t I = Pt.ci[e];
      for (int32_t a = A.rp[I]; a < A.rp[I + 1]; ++a) {
        const int32_t k = A.ci[a];
        s += P.rp[k + 1] - P.rp[k];
      }
    }
    return s;
  }
};

// Rows of A B (row-wise product, Alg. 1): r -> k in A(r,:) -> j in B(k,:).
struct Expand2 {
  CsrI A, B;
  template <class F>
  __device__ void run(int32_t row, int lane, int nl, const volatile int32_t* stop, F&& f) const {
    const int32_t a1 = A.rp[row + 1];
    for (int32_t a = A.rp[row] + lane; a < a1; a += nl) {
      const int32_t k = A.ci[a];
      const int32_t b1 = B.rp[k + 1];
      for (int32_t b = B.rp[k]; b < b1; ++b) {
        if (*stop) return;
        f(B.ci[b]);
      }
    }
  }
  __device__ int64_t bound(int32_t row) const {
    int64_t s = 0;
    for (int32_t a = A.rp[row]; a < A.rp[row + 1]; ++a) {
      const int32_t k = A.ci[a];
      s += B.rp[k + 1] - B.rp[k];
    }
    return s;
  }
};

// Bounded open-addressing insert of key j into a power-of-two table.
// Returns 1 if inserted, 0 if already present, -1 if the table is full.
__device__ __forceinline__ int set_insert(int32_t* keys, int cap_log2, int32_t j) {
  const uint32_t mask = (1u << cap_log2) - 1u;
  uint32_t h = hash32((uint32_t)j) >> (32 - cap_log2);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t cur = ((volatile int32_t*)keys)[h];
    if (cur == j) return 0;
    if (cur == kEmpty) {
      const int32_t old = atomicCAS(&keys[h], kEmpty, j);
      if (old == kEmpty) return 1;
      if (old == j) return 0;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

// Warp-wide ascending bitonic sort of n entries of shared memory keys.
__device__ void warp_bitonic(int32_t* k, int n, int lane) {
  int p = 1;
  while (p < n) p <<= 1;
  for (int size = 2; size <= p; size <<= 1) {
    for (int j = size >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < (p >> 1); t += 32) {
        int a, b;
        if (j == (size >> 1)) {
          a = (t / j) * size + (t % j);
          b = (t / j) * size + size - 1 - (t % j);
        } else {
          a = (t / j) * 2 * j + (t % j);
          b = a + j;
        }
        if (b < n) {
          const int32_t ka = k[a], kb = k[b];
          if (ka > kb) {
            k[a] = kb;
            k[b] = ka;
          }
        }
      }
      __syncwarp();
    }
  }
}

__device__ void cta_bitonic_keys(int32_t* k, int n) {
  int p = 1;
  while (p < n) p <<= 1;
  for (int size = 2; size <= p; size <<= 1) {
    for (int j = size >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (p >> 1); t += blockDim.x) {
        int a, b;
        if (j == (size >> 1)) {
          a = (t / j) * size + (t % j);
          b = (t / j) * size + size - 1 - (t % j);
        } else {
          a = (t / j) * 2 * j + (t % j);
          b = a + j;
        }
        if (b < n) {
          const int32_t ka = k[a], kb = k[b];
          if (ka > kb) {
            k[a] = kb;
            k[b] = ka;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Write the `count` keys of a warp table (cap slots, empty = kEmpty) to out,
// ascending.  tmp is 32 ints of warp-private shared memory.
__device__ void warp_emit_sorted(int32_t* keys, int cap, int count, int32_t* tmp,
                                 int32_t* out, int lane) {
  if (count <= 32) {
    int off = 0;
    for (int base = 0; base < cap; base += 32) {
      const int32_t key = keys[base + lane];
      const bool valid = key != kEmpty;
      const unsigned m = __ballot_sync(0xffffffffu, valid);
      if (valid) tmp[off + __popc(m & ((1u << lane) - 1u))] = key;
      off += __popc(m);
    }
    __syncwarp();
    int32_t k = lane < count ? tmp[lane] : kEmpty;
    for (int size = 2; size <= 32; size <<= 1) {
      for (int j = size >> 1; j > 0; j >>= 1) {
        const int partner = (j == (size >> 1)) ? (lane ^ (size - 1)) : (lane ^ j);
        const int32_t pk = __shfl_sync(0xffffffffu, k, partner);
        if (lane < partner ? (pk < k) : (pk > k)) k = pk;
      }
    }
    if (lane < count) out[lane] = k;
  } else {
    warp_bitonic(keys, cap, lane);
    for (int t = lane; t < count; t += 32) out[t] = keys[t];
  }
  __syncwarp();
}

// Tier 0: one warp per row, a private table of 2^cap_log2 slots in shared
// memory.  Rows whose distinct count exceeds `limit` go to tier 1.
// With `stash` (count pass only), a row of at most 32 columns also leaves
// them sorted in stash[32 row ..] and is marked tier 3: the fill pass then
// copies it instead of expanding the row a second time.
template <class E, bool FILL>
__global__ void k_union_warp(E ex, int32_t nrows, int cap_log2, int limit, uint8_t* tier,
                             int32_t* cnt, const int32_t* __restrict__ out_rp, int32_t* out_ci,
                             int32_t* ovf_list, int32_t* ovf_count, int32_t* stash) {
  extern __shared__ int32_t sm[];
  __shared__ int32_t wcount[32];
  __shared__ int32_t wflag[32];
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = 1 << cap_log2;
  int32_t* keys = sm + w * (cap + 32);
  int32_t* tmp = keys + cap;
  for (int64_t r = (int64_t)blockIdx.x * warps + w; r < nrows; r += (int64_t)gridDim.x * warps) {
    const int32_t row = (int32_t)r;
    if (FILL && tier[row] != 0) continue;
    for (int s = lane; s < cap; s += 32) keys[s] = kEmpty;
    if (lane == 0) {
      wcount[w] = 0;
      wflag[w] = 0;
    }
    __syncwarp();
    ex.run(row, lane, 32, &wflag[w], [&](int32_t j) {
      const int ins = set_insert(keys, cap_log2, j);
      if (ins == 1) {
        if (atomicAdd(&wcount[w], 1) + 1 > limit) wflag[w] = 1;
      } else if (ins < 0) {
        wflag[w] = 1;
      }
    });
    __syncwarp();
    const int count = ((volatile int32_t*)wcount)[w];
    const int ovf = ((volatile int32_t*)wflag)[w];
    if (!FILL) {
      const bool stashed = stash && !ovf && count <= 32;
      if (stashed) warp_emit_sorted(keys, cap, count, tmp, stash + (int64_t)row * 32, lane);
      if (lane == 0) {
        if (ovf) {
          tier[row] = 1;
          cnt[row] = 0;
          ovf_list[atomicAdd(ovf_count, 1)] = row;
        } else {
          tier[row] = stashed ? 3 : 0;
          cnt[row] = count;
        }
      }
    } else {
      warp_emit_sorted(keys, cap, count, tmp, out_ci + out_rp[row], lane);
    }
    __syncwarp();
  }
}

// Fill pass of the stashed rows: their sorted columns to their place in C.
__global__ void k_unstash(int32_t nrows, const uint8_t* __restrict__ tier, const int32_t* __restrict__ stash,
                          const int32_t* __restrict__ out_rp, int32_t* out_ci) {
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int64_t r = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); r < nrows; r += (int64_t)gridDim.x * warps) {
    if (tier[r] != 3) continue;
    const int32_t b = out_rp[r], len = out_rp[r + 1] - b;
    if (lane < len) out_ci[b + lane] = stash[r * 32 + lane];
  }
}

// Tier 1: one CTA per listed row, a table of 2^cap_log2 slots in shared memory.
template <class E, bool FILL>
__global__ void k_union_cta(E ex, const int32_t* __restrict__ list, int32_t nlist, int cap_log2,
                            int limit, uint8_t* tier, int32_t* cnt, const int32_t* __restrict__ out_rp,
                            int32_t* out_ci, int32_t* ovf_list, int32_t* ovf_count) {
  extern __shared__ int32_t keys[];
  __shared__ int32_t count, flag;
  const int cap = 1 << cap_log2;
  for (int32_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t row = list[li];
    if (FILL && tier[row] != 1) continue;  // block-uniform
    for (int s = threadIdx.x; s < cap; s += blockDim.x) keys[s] = kEmpty;
    if (threadIdx.x == 0) {
      count = 0;
      flag = 0;
    }
    __syncthreads();
    ex.run(row, threadIdx.x, blockDim.x, &flag, [&](int32_t j) {
      const int ins = set_insert(keys, cap_log2, j);
      if (ins == 1) {
        if (atomicAdd(&count, 1) + 1 > limit) flag = 1;
      } else if (ins < 0) {
        flag = 1;
      }
    });
    __syncthreads();
    const int c = count;
    if (!FILL) {
      if (threadIdx.x == 0) {
        if (flag) {
          tier[row] = 2;
          cnt[row] = 0;
          ovf_list[atomicAdd(ovf_count, 1)] = row;
        } else {
          tier[row] = 1;
          cnt[row] = c;
        }
      }
    } else {
      cta_bitonic_keys(keys, cap);
      int32_t* out = out_ci + out_rp[row];
      for (int t = threadIdx.x; t < c; t += blockDim.x) out[t] = keys[t];
    }
    __syncthreads();
  }
}

// Tier 2 bound: capacity of each spilled row's global table.
template <class E>
__global__ void k_spill_bound(E ex, const int32_t* __restrict__ list, int32_t nlist, int64_t ncols,
                              int64_t* cap) {
  const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= nlist) return;
  int64_t ub = ex.bound(list[li]);
  if (ub > ncols) ub = ncols;
  int64_t c = 64;
  while (c < 2 * ub) c <<= 1;
  cap[li] = c;
}

// Tier 2: one CTA per spilled row, a table in global memory (arena slice).
// The count pass leaves the keys in place; the fill pass sorts them there.
template <class E>
__global__ void k_union_global(E ex, const int32_t* __restrict__ list, int32_t nlist,
                               const int64_t* __restrict__ off, int32_t* arena, int32_t* cnt,
                               int32_t* status) {
  __shared__ int32_t count, flag;
  for (int32_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t row = list[li];
    const int64_t cap = off[li + 1] - off[li];
    const int cap_log2 = ilog2_ceil((uint32_t)cap);
    int32_t* keys = arena + off[li];
    for (int64_t s = threadIdx.x; s < cap; s += blockDim.x) keys[s] = kEmpty;
    if (threadIdx.x == 0) {
      count = 0;
      flag = 0;
    }
    __syncthreads();
    ex.run(row, threadIdx.x, blockDim.x, &flag, [&](int32_t j) {
      const int ins = set_insert(keys, cap_log2, j);
      if (ins == 1) atomicAdd(&count, 1);
      else if (ins < 0) flag = 1;
    });
    __syncthreads();
    if (threadIdx.x == 0) {
      cnt[row] = count;
      if (flag) atomicExch(status, PTAP_ERR_SPILL);
    }
    __syncthreads();
  }
}

__global__ void k_emit_global(const int32_t* __restrict__ list, int32_t nlist,
                              const int64_t* __restrict__ off, int32_t* arena,
                              const int32_t* __restrict__ out_rp, int32_t* out_ci) {
  for (int32_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t row = list[li];
    const int64_t cap = off[li + 1] - off[li];
    int32_t* keys = arena + off[li];
    cta_bitonic_keys(keys, (int)cap);
    const int32_t b = out_rp[row], c = out_rp[row + 1] - b;
    for (int t = threadIdx.x; t < c; t += blockDim.x) out_ci[b + t] = keys[t];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// pattern union driver shared by the all-at-once and two-step symbolic phases
// ---------------------------------------------------------------------------
struct UnionTiers {
  int warp_log2 = 8, warp_limit = 192;
  int cta_log2 = 13, cta_limit = 6144;
  int spilled = 0;
};

static UnionTiers tiers_for(const Config& cfg) {
  UnionTiers t;
  if (cfg.force_spill) {
    t.warp_log2 = 5;
    t.warp_limit = 4;
    t.cta_log2 = 6;
    t.cta_limit = 12;
  }
  return t;
}

// Computes the pattern rows of an expansion: row pointer (nrows+1), column
// indices (allocated here in `mem`, returned in *ci), total in *nnz.
template <class E>
static int union_pattern(Tracker& mem, const E& ex, int32_t nrows, int32_t ncols,
                         const Config& cfg, int32_t* rp, int32_t** ci, int64_t* nnz,
                         int32_t* status, int* spilled_rows, cudaStream_t s) {
  UnionTiers t = tiers_for(cfg);
  Scratch sc(&mem);
  int32_t *cnt = nullptr, *l1 = nullptr, *l2 = nullptr, *ctr = nullptr;
  uint8_t* tier = nullptr;
  PTAP_TRY(sc.get(&cnt, (int64_t)nrows + 1));
  PTAP_TRY(sc.get(&tier, nrows));
  PTAP_TRY(sc.get(&ctr, 2));
  PTAP_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(int32_t), s));
  const int threads = 256, warps = threads / 32;
  const size_t warp_smem = (size_t)warps * ((1 << t.warp_log2) + 32) * sizeof(int32_t);
  const int grid_w = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nrows, warps),
                                                                 (int64_t)num_sms() * 16));
  const size_t cta_smem = (size_t)(1 << t.cta_log2) * sizeof(int32_t);
  PTAP_TRY(grow_smem_limit((const void*)k_union_cta<E, false>, (int)cta_smem));
  PTAP_TRY(grow_smem_limit((const void*)k_union_cta<E, true>, (int)cta_smem));
  // --- count pass (rows of at most 32 columns also keep them in a stash, when
  //     the 128 bytes a row fit: the fill pass then only copies those rows)
  PTAP_TRY(sc.get(&l1, std::max<int64_t>(nrows, 1)));
  PhaseRange r_count("ptap: union count pass", s);
  int32_t* stash = nullptr;
  if (nrows > 0 && (int64_t)nrows * 128 <= ((int64_t)2 << 30) && mem.get_n(&stash, (int64_t)nrows * 32) != PTAP_OK)
    stash = nullptr;
  if (nrows > 0) {
    k_union_warp<E, false><<<grid_w, threads, warp_smem, s>>>(ex, nrows, t.warp_log2, t.warp_limit,
                                                               tier, cnt, nullptr, nullptr, l1, ctr, stash);
    PTAP_LAUNCHED();
  }
  int32_t h_ctr[2] = {0, 0};
  PTAP_CUDA(cudaMemcpyAsync(h_ctr, ctr, sizeof(h_ctr), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  const int32_t n1 = h_ctr[0];
  int32_t n2 = 0;
  if (n1 > 0) {
    PTAP_TRY(sc.get(&l2, n1));
    const int grid = (int)std::min<int64_t>(n1, (int64_t)num_sms() * 4);
    k_union_cta<E, false><<<grid, threads, cta_smem, s>>>(ex, l1, n1, t.cta_log2, t.cta_limit, tier,
                                                          cnt, nullptr, nullptr, l2, ctr + 1);
    PTAP_LAUNCHED();
    PTAP_CUDA(cudaMemcpyAsync(&n2, ctr + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
  }
  int64_t* off = nullptr;
  int32_t* arena = nullptr;
  if (n2 > 0) {
    int64_t* capd = nullptr;
    PTAP_TRY(sc.get(&capd, n2));
    PTAP_TRY(sc.get(&off, (int64_t)n2 + 1));
    k_spill_bound<E><<<(unsigned)ceil_div(n2, 128), 128, 0, s>>>(ex, l2, n2, ncols, capd);
    PTAP_LAUNCHED();
    std::vector<int64_t> hcap(n2), hoff(n2 + 1, 0);
    PTAP_CUDA(cudaMemcpyAsync(hcap.data(), capd, n2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
    for (int32_t i = 0; i < n2; ++i) {
      if (hcap[i] > ((int64_t)1 << 30)) return PTAP_ERR_OVERFLOW;
      hoff[i + 1] = hoff[i] + hcap[i];
    }
    PTAP_CUDA(cudaMemcpyAsync(off, hoff.data(), (n2 + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    PTAP_TRY(sc.get(&arena, hoff[n2]));
    const int grid = (int)std::min<int64_t>(n2, (int64_t)num_sms() * 2);
    k_union_global<E><<<grid, 256, 0, s>>>(ex, l2, n2, off, arena, cnt, status);
    PTAP_LAUNCHED();
  }
  if (spilled_rows) *spilled_rows = n2;
  // --- preallocate: exclusive scan of the counts
  int64_t total = 0;
  PTAP_TRY(exclusive_scan(mem, cnt, rp, nrows, &total, s));
  *nnz = total;
  PTAP_TRY(mem.get_n(ci, total));
  // --- fill pass
  PhaseRange r_fill("ptap: union fill pass", s);
  if (nrows > 0) {
    k_union_warp<E, true><<<grid_w, threads, warp_smem, s>>>(ex, nrows, t.warp_log2, t.warp_limit,
                                                              tier, cnt, rp, *ci, nullptr, nullptr, nullptr);
    PTAP_LAUNCHED();
    if (stash) {
      k_unstash<<<grid_w, threads, 0, s>>>(nrows, tier, stash, rp, *ci);
      PTAP_LAUNCHED();
      mem.put(stash);
    }
  }
  if (n1 > 0) {
    const int grid = (int)std::min<int64_t>(n1, (int64_t)num_sms() * 4);
    k_union_cta<E, true><<<grid, threads, cta_smem, s>>>(ex, l1, n1, t.cta_log2, t.cta_limit, tier,
                                                         cnt, rp, *ci, nullptr, nullptr);
    PTAP_LAUNCHED();
  }
  if (n2 > 0) {
    const int grid = (int)std::min<int64_t>(n2, (int64_t)num_sms() * 2);
    k_emit_global<<<grid, 256, 0, s>>>(l2, n2, off, arena, rp, *ci);
    PTAP_LAUNCHED();
  }
  return PTAP_OK;
}

// Explicit instantiation entry for the two-step symbolic (row-wise A B).
int union_pattern_ab(Tracker& mem, const CsrI& A, const CsrI& B, const Config& cfg, int32_t* rp,
                     int32_t** ci, int64_t* nnz, int32_t* status, int* spilled, cudaStream_t s) {
  Expand2 ex{A, B};
  return union_pattern(mem, ex, A.nrows, B.ncols, cfg, rp, ci, nnz, status, spilled, s);
}

// ---------------------------------------------------------------------------
// input checks
// ---------------------------------------------------------------------------
int check_csr_host(const ptap_csr* M, bool need_val) {
  if (!M) return PTAP_ERR_INVALID;
  if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0 || M->nnz >= ((int64_t)1 << 31))
    return PTAP_ERR_INVALID;
  if (M->dtype != PTAP_F64 && M->dtype != PTAP_F32) return PTAP_ERR_INVALID;
  if (!M->row_ptr) return PTAP_ERR_INVALID;
  if (M->nnz > 0 && !M->col_idx) return PTAP_ERR_INVALID;
  if (need_val && M->nnz > 0 && !M->val) return PTAP_ERR_INVALID;
  return PTAP_OK;
}

namespace {
__global__ void k_validate(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           int32_t nrows, int32_t ncols, int64_t nnz, int32_t* bad) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int32_t b = rp[r], e = rp[r + 1];
  if (r == 0 && b != 0) atomicExch(bad, 1);
  if (r == nrows - 1 && (int64_t)e != nnz) atomicExch(bad, 1);
  if (b > e || b < 0 || (int64_t)e > nnz) {
    atomicExch(bad, 1);
    return;
  }
  int32_t prev = -1;
  for (int32_t x = b; x < e; ++x) {
    const int32_t c = ci[x];
    if (c < 0 || c >= ncols || c <= prev) {
      atomicExch(bad, 1);
      return;
    }
    prev = c;
  }
}
}  // namespace

int validate_csr(Tracker& mem, const ptap_csr* M, cudaStream_t s) {
  Scratch sc(&mem);
  int32_t* bad = nullptr;
  PTAP_TRY(sc.get(&bad, 1));
  PTAP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  if (M->nrows > 0) {
    k_validate<<<(unsigned)ceil_div(M->nrows, 256), 256, 0, s>>>(M->row_ptr, M->col_idx, M->nrows,
                                                                 M->ncols, M->nnz, bad);
    PTAP_LAUNCHED();
  }
  int32_t h = 0;
  PTAP_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  return h ? PTAP_ERR_INVALID : PTAP_OK;
}

// row_ptr[0] == 0 and row_ptr[nrows] == nnz, read back (synchronises).
static int check_ends(const ptap_csr* M, cudaStream_t s) {
  int32_t h[2] = {0, 0};
  PTAP_CUDA(cudaMemcpyAsync(&h[0], M->row_ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaMemcpyAsync(&h[1], M->row_ptr + M->nrows, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  if (h[0] != 0 || (int64_t)h[1] != M->nnz) return PTAP_ERR_INVALID;
  return PTAP_OK;
}

// ---------------------------------------------------------------------------
// transpose of a pattern (count, scan, scatter, sort each column)
// ---------------------------------------------------------------------------
namespace {
__global__ void k_col_count(const int32_t* __restrict__ ci, int64_t nnz, int32_t* cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[e]], 1);
}
__global__ void k_col_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           int32_t nrows, const int32_t* __restrict__ tp, int32_t* cursor,
                           int32_t* tj, int32_t* tperm) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    for (int32_t e = rp[r]; e < rp[r + 1]; ++e) {
      const int32_t c = ci[e];
      const int32_t dst = tp[c] + atomicAdd(&cursor[c], 1);
      tj[dst] = (int32_t)r;
      if (tperm) tperm[dst] = e;
    }
  }
}
}  // namespace

int transpose_pattern(Tracker& mem, const CsrI& M, int32_t* tp, int32_t* tj, int32_t* tperm,
                      cudaStream_t s) {
  Scratch sc(&mem);
  int32_t* cnt = nullptr;
  PTAP_TRY(sc.get(&cnt, (int64_t)M.ncols + 1));
  PTAP_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)M.ncols + 1) * sizeof(int32_t), s));
  int32_t nnz_h = 0;
  PTAP_CUDA(cudaMemcpyAsync(&nnz_h, M.rp + M.nrows, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  const int grid = num_sms() * 8;
  if (nnz_h > 0) {
    k_col_count<<<grid, 256, 0, s>>>(M.ci, nnz_h, cnt);
    PTAP_LAUNCHED();
  }
  int64_t total = 0;
  PTAP_TRY(exclusive_scan(mem, cnt, tp, M.ncols, &total, s));
  PTAP_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)M.ncols + 1) * sizeof(int32_t), s));
  if (M.nrows > 0) {
    k_col_fill<<<grid, 256, 0, s>>>(M.rp, M.ci, M.nrows, tp, cnt, tj, tperm);
    PTAP_LAUNCHED();
  }
  return segmented_sort(mem, tp, M.ncols, tj, tperm, -1, s);
}

// ---------------------------------------------------------------------------
// owner-mode schedule: coarse rows cut into chunks whose C entries fit on
// chip, and for each chunk the ascending list of fine rows I whose P(I,:)
// reaches into it.  Fine rows with an empty P(I,:) contribute nothing and are
// never visited (Alg. 7-8 skip them).
// ---------------------------------------------------------------------------
namespace {
__global__ void k_row_chunk(const int32_t* __restrict__ chunk_row, int32_t nchunks, int32_t m,
                            int32_t* row_chunk) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = nchunks - 1;  // last chunk c with chunk_row[c] <= i
    while (lo < hi) {
      const int32_t mid = (lo + hi + 1) >> 1;
      if (chunk_row[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    row_chunk[i] = lo;
  }
}
// For each fine row, the distinct chunks among its (sorted) P columns.  With
// ranges of rows a chunk's columns are consecutive, so comparing with the
// previous one suffices.  With compact chunks (ANY) a chunk may recur after
// another, so each column is compared with all earlier ones of the row; rows
// longer than kMaxAny set *too_long and are skipped (the caller then falls
// back to ranges: such rows never run class programs).  Neighbouring fine
// rows mostly reach the same chunks, so the lanes of a warp that add to one
// chunk's count take their slots with a single atomic.  Loop bounds are
// uniform over the warp, so every lane reaches each match.
constexpr int kMaxAny = 8;
template <bool FILL, bool ANY>
__global__ void k_chunk_visits(const int32_t* __restrict__ Prp, const int32_t* __restrict__ Pci,
                               int32_t n, const int32_t* __restrict__ row_chunk, int32_t* cnt,
                               const int32_t* __restrict__ fptr, int32_t* frows, int32_t* too_long) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = b + threadIdx.x;
    int32_t e0 = 0, len = 0;
    if (I < n) {
      e0 = Prp[I];
      len = Prp[I + 1] - e0;
    }
    if (ANY && len > kMaxAny) {
      atomicExch(too_long, 1);
      len = 0;
    }
    const int32_t maxlen = __reduce_max_sync(0xffffffffu, len);
    int32_t prev = -1;
    for (int32_t x = 0; x < maxlen; ++x) {
      int32_t c = -1;
      if (x < len) {
        c = row_chunk[Pci[e0 + x]];
        bool fresh = c != prev;
        if (ANY)
          for (int32_t d = 0; d < x && fresh; ++d) fresh = row_chunk[Pci[e0 + d]] != c;
        if (fresh) prev = c;
        else c = -1;
      }
      const unsigned peers = __match_any_sync(0xffffffffu, c);
      if (c >= 0) {
        const int leader = __ffs(peers) - 1;
        int32_t slot = 0;
        if (lane == leader) slot = atomicAdd(&cnt[c], __popc(peers));
        slot = __shfl_sync(peers, slot, leader) + __popc(peers & ((1u << lane) - 1u));
        if (FILL) frows[fptr[c] + slot] = (int32_t)I;
      }
    }
  }
}
}  // namespace

// Visit lists of the chunks given row_chunk (chunk of every coarse row):
// counts, offsets chunk_fptr, fine rows chunk_frows ascending per chunk.
// *too_long is set (and nothing built) when ANY and a row of P is longer than
// kMaxAny.
template <bool ANY>
static int build_visits(ptap_plan* p, const ptap_csr* P, const int32_t* row_chunk, bool* too_long,
                        cudaStream_t s) {
  const int32_t nch = p->nchunks;
  Scratch sc(&p->mem);
  int32_t* cnt = nullptr;
  PTAP_TRY(sc.get(&cnt, (int64_t)nch + 2));
  int32_t* flag = cnt + nch + 1;
  const int grid = num_sms() * 8;
  PTAP_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)nch + 2) * sizeof(int32_t), s));
  if (p->n > 0) {
    k_chunk_visits<false, ANY><<<grid, 256, 0, s>>>(P->row_ptr, P->col_idx, p->n, row_chunk, cnt, nullptr,
                                                    nullptr, flag);
    PTAP_LAUNCHED();
  }
  *too_long = false;
  if (ANY) {
    int32_t f = 0;
    PTAP_CUDA(cudaMemcpyAsync(&f, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
    if (f) {
      *too_long = true;
      return PTAP_OK;
    }
  }
  int64_t total = 0;
  PTAP_TRY(p->mem.get_n(&p->chunk_fptr, (int64_t)nch + 1));
  PTAP_TRY(exclusive_scan(p->mem, cnt, p->chunk_fptr, nch, &total, s));
  p->nfrows = total;
  PTAP_TRY(p->mem.get_n(&p->chunk_frows, total));
  PTAP_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)nch + 1) * sizeof(int32_t), s));
  if (p->n > 0) {
    k_chunk_visits<true, ANY><<<grid, 256, 0, s>>>(P->row_ptr, P->col_idx, p->n, row_chunk, cnt,
                                                   p->chunk_fptr, p->chunk_frows, flag);
    PTAP_LAUNCHED();
  }
  return segmented_sort(p->mem, p->chunk_fptr, nch, p->chunk_frows, nullptr, -1, s);
}

static int build_schedule(ptap_plan* p, const ptap_csr* P, cudaStream_t s) {
  const int32_t m = p->m;
  const int CH = p->cfg.chunk_entries;
  const int MAXR = 2048;
  std::vector<int32_t> rp(m + 1);
  PTAP_CUDA(cudaMemcpyAsync(rp.data(), p->c_rp, (m + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> cr;
  int32_t i = 0, heavy = 0, max_rows = 0, max_nnz = 0;
  while (i < m) {
    cr.push_back(i);
    const int32_t b = rp[i];
    int32_t j = i;
    if (rp[i + 1] - b > CH) {
      j = i + 1;
      ++heavy;
    } else {
      while (j < m && rp[j + 1] - b <= CH && j - i < MAXR) ++j;
    }
    max_rows = std::max(max_rows, j - i);
    if (rp[i + 1] - b <= CH) max_nnz = std::max(max_nnz, rp[j] - b);
    i = j;
  }
  const int32_t nch = (int32_t)cr.size();
  cr.push_back(m);
  p->nchunks = nch;
  p->nheavy = heavy;
  p->max_chunk_rows = max_rows;
  p->max_chunk_nnz = max_nnz;
  PTAP_TRY(p->mem.get_n(&p->chunk_row, (int64_t)nch + 1));
  PTAP_CUDA(cudaMemcpyAsync(p->chunk_row, cr.data(), cr.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  if (nch == 0) {
    PTAP_TRY(p->mem.get_n(&p->chunk_fptr, 1));
    PTAP_CUDA(cudaMemsetAsync(p->chunk_fptr, 0, sizeof(int32_t), s));
    PTAP_TRY(p->mem.get_n(&p->chunk_frows, 1));
    p->nfrows = 0;
    return PTAP_OK;
  }
  Scratch sc(&p->mem);
  int32_t* row_chunk = nullptr;
  PTAP_TRY(sc.get(&row_chunk, m));
  k_row_chunk<<<num_sms() * 8, 256, 0, s>>>(p->chunk_row, nch, m, row_chunk);
  PTAP_LAUNCHED();
  bool unused = false;
  return build_visits<false>(p, P, row_chunk, &unused, s);
}

// Compact chunks: regions of the graph of C's pattern (row i adjacent to the
// columns of C(i,:)), grown breadth-first over runs of L consecutive coarse
// rows (L = compact_chunks) from the lowest run not yet taken, until the next
// run reached would overflow the chunk.  On a mesh the regions are blocks of
// coarse points instead of slabs, so fewer fine rows have P(I,:) entries in
// two chunks (each such visit recomputes the row of A P); runs keep a warp's
// fine rows, which lie along the fastest-varying index, on one line of the
// block.  Sets *done when the plan's schedule was built this way; leaves the
// plan untouched otherwise (a run longer than a chunk, too many chunks for
// the packed locations, or a P row too long for the visit lists).
static int build_schedule_compact(ptap_plan* p, const ptap_csr* P, cudaStream_t s, bool* done) {
  *done = false;
  const int32_t m = p->m;
  const int CH = p->cfg.chunk_entries;
  if (m == 0 || p->nnz_c == 0) return PTAP_OK;
  std::vector<int32_t> rp(m + 1), ci(p->nnz_c);
  PTAP_CUDA(cudaMemcpyAsync(rp.data(), p->c_rp, (m + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaMemcpyAsync(ci.data(), p->c_ci, ci.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  const int32_t L = std::max(1, p->cfg.compact_chunks);
  const int32_t nruns = (int32_t)(((int64_t)m + L - 1) / L);
  auto run_nnz = [&](int32_t r) { return rp[std::min<int64_t>((int64_t)(r + 1) * L, m)] - rp[(int64_t)r * L]; };
  for (int32_t r = 0; r < nruns; ++r)
    if (run_nnz(r) > CH) return PTAP_OK;
  int loc_bits = 1;
  while ((1 << loc_bits) < CH) ++loc_bits;
  // grow the regions, a run at a time
  std::vector<int32_t> own_run(nruns, -1), queue(nruns);
  int32_t nch = 0;
  for (int32_t seed = 0; seed < nruns; ++seed) {
    if (own_run[seed] >= 0) continue;
    int64_t head = 0, tail = 0, used = run_nnz(seed);
    own_run[seed] = nch;
    queue[tail++] = seed;
    bool full = false;
    while (head < tail && !full) {
      const int32_t q = queue[head++];
      const int32_t i1 = (int32_t)std::min<int64_t>((int64_t)(q + 1) * L, m);
      for (int32_t e = rp[(int64_t)q * L]; e < rp[i1] && !full; ++e) {
        const int32_t r = ci[e] / L;
        if (own_run[r] >= 0) continue;
        const int32_t len = run_nnz(r);
        if (used + len > CH) {
          full = true;
          break;
        }
        own_run[r] = nch;
        used += len;
        queue[tail++] = r;
      }
    }
    ++nch;
  }
  std::vector<int32_t> own(m);
  for (int32_t i = 0; i < m; ++i) own[i] = own_run[i / L];
  if ((int64_t)nch >= ((int64_t)1 << (31 - loc_bits))) return PTAP_OK;
  // rows of each chunk ascending, their accumulator offsets, the packed locations
  std::vector<int32_t> start(nch + 1, 0), nnz(nch, 0), crows(m), loc(m);
  for (int32_t i = 0; i < m; ++i) ++start[own[i] + 1];
  for (int32_t c = 0; c < nch; ++c) start[c + 1] += start[c];
  {
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int32_t i = 0; i < m; ++i) {
      const int32_t c = own[i];
      crows[fill[c]++] = i;
      loc[i] = (c << loc_bits) | nnz[c];
      nnz[c] += rp[i + 1] - rp[i];
    }
  }
  int32_t max_nnz = 0;
  for (int32_t c = 0; c < nch; ++c) max_nnz = std::max(max_nnz, nnz[c]);
  Scratch sc(&p->mem);
  int32_t* row_chunk = nullptr;
  PTAP_TRY(sc.get(&row_chunk, m));
  PTAP_CUDA(cudaMemcpyAsync(row_chunk, own.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  p->nchunks = nch;
  p->nheavy = 0;
  p->max_chunk_rows = 0;  // no row offsets on chip
  p->max_chunk_nnz = max_nnz;
  bool too_long = false;
  PTAP_TRY(build_visits<true>(p, P, row_chunk, &too_long, s));
  if (too_long) {
    p->nchunks = 0;
    return PTAP_OK;
  }
  PTAP_TRY(p->mem.get_n(&p->chunk_row, (int64_t)nch + 1));
  PTAP_TRY(p->mem.get_n(&p->chunk_crows, m));
  PTAP_TRY(p->mem.get_n(&p->row_loc, m));
  PTAP_TRY(p->mem.get_n(&p->chunk_nnz, nch));
  PTAP_CUDA(cudaMemcpyAsync(p->chunk_row, start.data(), start.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaMemcpyAsync(p->chunk_crows, crows.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaMemcpyAsync(p->row_loc, loc.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaMemcpyAsync(p->chunk_nnz, nnz.data(), nch * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  p->loc_bits = loc_bits;
  p->compact = true;
  *done = true;
  return PTAP_OK;
}

// Drops the owner-mode schedule (to rebuild it another way).
static void drop_schedule(ptap_plan* p) {
  int32_t** arrays[] = {&p->chunk_row, &p->chunk_fptr, &p->chunk_frows, &p->chunk_crows, &p->row_loc,
                        &p->chunk_nnz};
  for (int32_t** a : arrays) {
    if (*a) p->mem.put(*a);
    *a = nullptr;
  }
  p->compact = false;
  p->loc_bits = 0;
  p->nchunks = 0;
  p->nfrows = 0;
}

// ---------------------------------------------------------------------------
// common front half of both symbolic entry points
// ---------------------------------------------------------------------------
int symbolic_prologue(const ptap_csr* A, const ptap_csr* P, const ptap_config* cfg,
                      const ptap_allocator* alloc, void* stream, ptap_plan** out, int kind) {
  if (!out) return PTAP_ERR_INVALID;
  *out = nullptr;
  PTAP_TRY(check_csr_host(A, false));
  PTAP_TRY(check_csr_host(P, false));
  if (A->nrows != A->ncols || A->ncols != P->nrows || A->dtype != P->dtype) return PTAP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  ptap_plan* p = new (std::nothrow) ptap_plan();
  if (!p) return PTAP_ERR_OOM;
  p->kind = kind;
  p->dtype = A->dtype;
  p->n = A->nrows;
  p->m = P->ncols;
  p->nnz_a = A->nnz;
  p->nnz_p = P->nnz;
  p->stream = s;
  p->cfg = resolve_config(cfg);
  if (kind != 0) {  // the two-step kernels: CTAs of at most 256 threads
    p->cfg.block_threads = std::min(p->cfg.block_threads, 256);
    if (p->cfg.chunk_entries > 16384) p->cfg.chunk_entries = 16384;
  }
  p->mem.init(alloc, s);
  int rc = check_ends(A, s);
  if (rc == PTAP_OK) rc = check_ends(P, s);
  if (rc == PTAP_OK && p->cfg.debug_checks) {
    rc = validate_csr(p->mem, A, s);
    if (rc == PTAP_OK) rc = validate_csr(p->mem, P, s);
  }
  if (rc == PTAP_OK) rc = p->mem.get_n(&p->status, 1);
  if (rc == PTAP_OK && cudaMemsetAsync(p->status, 0, sizeof(int32_t), s) != cudaSuccess)
    rc = PTAP_ERR_CUDA;
  if (rc != PTAP_OK) {
    p->mem.release_all();
    delete p;
    return rc;
  }
  *out = p;
  return PTAP_OK;
}

// Largest chunk (entries) whose accumulator, with room for the row offsets and
// program buffers, fits the device's opt-in shared memory; a multiple of 1024.
static int fast_chunk_limit(int vb) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 8192;
  }
  const int n = (optin - 32 * 1024) / vb;
  return std::max(1024, std::min(65536, n & ~1023));
}

static int symbolic_body(ptap_plan* p, const ptap_csr* A, const ptap_csr* P) {
  cudaStream_t s = p->stream;
  const int32_t m = p->m;
  PTAP_TRY(p->mem.get_n(&p->c_rp, (int64_t)m + 1));
  {
    Scratch sc(&p->mem);
    int32_t *tp = nullptr, *tj = nullptr;
    PTAP_TRY(sc.get(&tp, (int64_t)m + 1));
    PTAP_TRY(sc.get(&tj, p->nnz_p));
    CsrI Pi{P->nrows, P->ncols, P->row_ptr, P->col_idx};
    {
      PhaseRange r1("ptap: transpose of P's pattern", s);
      PTAP_TRY(transpose_pattern(p->mem, Pi, tp, tj, nullptr, s));
    }
    Expand3 ex{CsrI{m, P->nrows, tp, tj}, CsrI{A->nrows, A->ncols, A->row_ptr, A->col_idx}, Pi};
    int spilled = 0;
    PhaseRange range("ptap: pattern of C", s);
    PTAP_TRY(union_pattern(p->mem, ex, m, m, p->cfg, p->c_rp, &p->c_ci, &p->nnz_c, p->status,
                           &spilled, s));
    p->spill_rows = spilled;
    PTAP_CUDA(cudaStreamSynchronize(s));
  }
  // Owner-mode schedule.  With per-class programs the on-chip accumulator
  // needs no column indices, so chunks can be larger (fewer fine rows are
  // visited by two chunks); without them the general kernel's default applies.
  // The class-program kernels accept CTAs of up to 1024 threads and chunks up
  // to 65536 entries (bounded by shared memory for the value type); the
  // general kernels keep at most 256 threads and 16384 entries.
  const bool user_ch = p->cfg.chunk_entries > 0;
  const int ch_fast = 8192, ch_general = 4096, ch_general_max = 16384;
  const int ch_fast_max = fast_chunk_limit(p->dtype == PTAP_F64 ? 8 : 4);
  const bool try_fast = p->cfg.class_programs && p->cfg.mode == PTAP_MODE_OWNER &&
                        !p->cfg.force_spill && (!user_ch || p->cfg.chunk_entries >= 256);
  const int user_value = p->cfg.chunk_entries;
  p->cfg.chunk_entries = user_ch ? std::min(user_value, try_fast ? ch_fast_max : ch_general_max)
                                 : (try_fast ? ch_fast : ch_general);
  {
    PhaseRange range("ptap: chunk schedule", s);
    bool compact = false;
    if (try_fast && p->cfg.compact_chunks) {
      PTAP_TRY(build_schedule_compact(p, P, s, &compact));
      if (!compact) drop_schedule(p);  // whatever a declined attempt left
    }
    if (!compact) PTAP_TRY(build_schedule(p, P, s));
  }
  if (try_fast) {
    PhaseRange range("ptap: structure classes", s);
    PTAP_TRY(build_classes(p, A, P, s));
    const int general_ch = user_ch ? std::min(user_value, ch_general_max) : ch_general;
    if (!p->fast && (p->cfg.chunk_entries != general_ch || p->compact)) {
      drop_schedule(p);
      p->cfg.chunk_entries = general_ch;
      PTAP_TRY(build_schedule(p, P, s));
    }
  }
  if (!p->fast) p->cfg.block_threads = std::min(p->cfg.block_threads, 256);
  PTAP_TRY(build_index_cache(p, A, P, s));
  {
    PhaseRange range("ptap: prepare numeric (code generation)", s);
    PTAP_TRY(prepare_numeric(p));
  }
  PTAP_CUDA(cudaStreamSynchronize(s));
  int32_t st = 0;
  PTAP_CUDA(cudaMemcpy(&st, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (st) return st;
  p->symbolic_peak = p->mem.peak;
  return PTAP_OK;
}

}  // namespace ptap

extern "C" int ptap_symbolic(const ptap_csr* A, const ptap_csr* P, const ptap_config* cfg,
                             const ptap_allocator* alloc, void* stream, ptap_plan** out) {
  ptap::Range range("ptap_symbolic");
  ptap_plan* p = nullptr;
  PTAP_TRY(ptap::symbolic_prologue(A, P, cfg, alloc, stream, &p, 0));
  int rc = ptap::symbolic_body(p, A, P);
  if (rc != PTAP_OK) {
    cudaStreamSynchronize(p->stream);
    p->mem.release_all();
    delete p;
    return rc;
  }
  *out = p;
  return PTAP_OK;
}
