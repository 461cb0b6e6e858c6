// General owner-mode numeric kernel, sort-based (the default general path).
//
// Same scheme as owner_chunk (owner.cuh): a CTA owns a chunk of coarse rows,
// zeroes an on-chip accumulator, visits the chunk's fine rows and writes the
// chunk's values once.  What differs is how a fine row's R = (A P)(I,:) is
// formed (Alg. 3) and added (Alg. 8).  Here one warp takes one fine row:
//
//  1. Lane a takes A(I,k_a) and its row P(k_a,:); the products A(I,k_a) P(k_a,b)
//     go to the warp's buffer in shared memory.
//  2. The products are sorted by column -- up to 32 in registers by a warp
//     bitonic sort, up to 256 in shared memory -- and a segmented scan over
//     equal columns sums them, so R's entries come out sorted, one per run.
//     No hash table, no probing, no atomics.
//  3. The pI x r terms P(I,i_s) R(t) are spread over the 32 lanes.  Each lane
//     finds its term's position in C's row i_s (a binary search over the
//     chunk's column indices in shared memory) and adds it.
//
// Rows with more than 256 products, more than 32 entries in A(I,:) or P(I,:),
// or chunks too heavy for shared memory take a direct path that adds every
// product A(I,k) P(k,j) P(I,i) without merging them first; it is correct for
// any row.  All lanes of a warp always take the same branch: the choices
// depend only on the row.
#include <algorithm>

#include "owner.cuh"

namespace ptap {

namespace {

constexpr int kRowMax = 256;  // products a warp sorts in shared memory

template <typename V>
struct SortedSmem {
  V* acc;
  int32_t* ccol;
  int32_t* roff;
  int32_t* wcol;  // per warp: kRowMax product columns (then R's, compacted in place)
  V* wval;        // per warp: kRowMax product values (then R's)
  int32_t* wi;    // per warp: 32 coarse rows of P(I,:)
  V* ww;          // per warp: 32 weights of P(I,:)
  __device__ SortedSmem(unsigned char* raw, int CH, int max_rows, int nwarps) {
    acc = (V*)raw;
    wval = acc + CH;
    ww = wval + (size_t)nwarps * kRowMax;
    ccol = (int32_t*)(ww + (size_t)nwarps * 32);
    roff = ccol + CH;
    wcol = roff + max_rows + 1;
    wi = wcol + (size_t)nwarps * kRowMax;
  }
};

template <typename V>
__device__ __forceinline__ void add_term(V* acc, const int32_t* col, int32_t lo, int32_t hi, int32_t j, V wv,
                                         bool on_chip, int32_t* status) {
  const int32_t pos = find_col(col, lo, hi, j);
  if (pos < 0) {
    atomicExch(status, PTAP_ERR_PATTERN);
    return;
  }
  atomicAdd(&acc[pos], wv);
  (void)on_chip;
}

// Every product A(I,k) P(k,j) times every P(I,i) with i in the chunk, without
// forming R: for rows the sorted path does not take.
template <typename V>
__device__ void direct_row(const NumArgs<V>& a, int32_t I, int32_t i0, int32_t i1, V* acc, const int32_t* col,
                           const int32_t* roff, bool on_chip) {
  const int lane = threadIdx.x & 31;
  const int32_t a0 = a.A.rp[I], a1 = a.A.rp[I + 1];
  const int32_t p0 = a.P.rp[I], p1 = a.P.rp[I + 1];
  for (int32_t x = a0 + lane; x < a1; x += 32) {
    const int32_t k = a.A.ci[x];
    const V av = a.A.val[x];
    for (int32_t b = a.P.rp[k]; b < a.P.rp[k + 1]; ++b) {
      const int32_t j = a.P.ci[b];
      const V t = av * a.P.val[b];
      for (int32_t e = p0; e < p1; ++e) {
        const int32_t i = a.P.ci[e];
        if (i < i0) continue;
        if (i >= i1) break;
        add_term(acc, col, roff[i - i0], roff[i - i0 + 1], j, a.P.val[e] * t, on_chip, a.status);
      }
    }
  }
}

template <typename V>
__device__ void sorted_chunk(const NumArgs<V>& a, int32_t c, SortedSmem<V>& sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int32_t i0 = a.chunk_row[c], i1 = a.chunk_row[c + 1];
  const int32_t base = a.c_rp[i0], nnz = a.c_rp[i1] - base;
  const bool on_chip = nnz <= a.CH;
  V* acc = on_chip ? sm.acc : a.c_val + base;
  const int32_t* col = on_chip ? sm.ccol : a.c_ci + base;
  if (on_chip) {
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) {
      sm.acc[t] = V(0);
      sm.ccol[t] = a.c_ci[base + t];
    }
  } else {
    for (int64_t t = threadIdx.x; t < nnz; t += blockDim.x) acc[t] = V(0);
  }
  for (int r = threadIdx.x; r <= i1 - i0; r += blockDim.x) sm.roff[r] = a.c_rp[i0 + r] - base;
  __syncthreads();
  int32_t* pcol = sm.wcol + warp * kRowMax;  // products, then R (compacted in place)
  V* pval = sm.wval + warp * kRowMax;
  int32_t* wi = sm.wi + warp * 32;
  V* ww = sm.ww + warp * 32;
  const int32_t f1 = a.chunk_fptr[c + 1];
  for (int32_t f = a.chunk_fptr[c] + warp; f < f1; f += nwarps) {
    const int32_t I = a.chunk_frows[f];
    const int32_t a0 = a.A.rp[I], na = a.A.rp[I + 1] - a0;
    const int32_t p0 = a.P.rp[I], pI = a.P.rp[I + 1] - p0;
    if (na > 32 || pI > 32 || !on_chip) {
      direct_row(a, I, i0, i1, acc, col, sm.roff, on_chip);
      continue;
    }
    // (1) products: lane a expands P(k_a,:)
    int32_t pb = 0, pa = 0;
    V av = V(0);
    if (lane < na) {
      const int32_t k = a.A.ci[a0 + lane];
      av = a.A.val[a0 + lane];
      pb = a.P.rp[k];
      pa = a.P.rp[k + 1] - pb;
    }
    int32_t off = pa;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, off, d);
      if (lane >= d) off += y;
    }
    const int32_t T = __shfl_sync(0xffffffffu, off, 31);
    if (T > kRowMax) {
      direct_row(a, I, i0, i1, acc, col, sm.roff, on_chip);
      continue;
    }
    off -= pa;
    for (int32_t b = 0; b < pa; ++b) {
      pcol[off + b] = a.P.ci[pb + b];
      pval[off + b] = av * a.P.val[pb + b];
    }
    if (lane < pI) {
      wi[lane] = a.P.ci[p0 + lane];
      ww[lane] = a.P.val[p0 + lane];
    }
    __syncwarp();
    int32_t r = 0;
    if (T <= 32) {
      // (2) sort the products by column in registers, then sum equal columns
      int32_t kc = lane < T ? pcol[lane] : INT32_MAX;
      V kv = lane < T ? pval[lane] : V(0);
#pragma unroll
      for (int k2 = 2; k2 <= 32; k2 <<= 1)
#pragma unroll
        for (int j = k2 >> 1; j > 0; j >>= 1) {
          const int32_t oc = __shfl_xor_sync(0xffffffffu, kc, j);
          const V ov = __shfl_xor_sync(0xffffffffu, kv, j);
          const bool keep_min = ((lane & j) == 0) == ((lane & k2) == 0);
          if (keep_min ? (oc < kc) : (oc > kc)) {
            kc = oc;
            kv = ov;
          }
        }
      V run = kv;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const V y = __shfl_up_sync(0xffffffffu, run, d);
        const int32_t cy = __shfl_up_sync(0xffffffffu, kc, d);
        if (lane >= d && cy == kc) run += y;
      }
      const int32_t next = __shfl_down_sync(0xffffffffu, kc, 1);
      const bool last = lane < T && (lane == 31 || next != kc);
      const unsigned lm = __ballot_sync(0xffffffffu, last);
      r = __popc(lm);
      __syncwarp();
      if (last) {
        const int32_t t = __popc(lm & ((1u << lane) - 1u));
        pcol[t] = kc;
        pval[t] = run;
      }
    } else {
      // (2') up to kRowMax products: bitonic sort of the pairs in shared
      // memory (padding to a power of two sorts last), then the runs of
      // equal columns are summed window by window, compacted in place
      int pw = 64, lp = 6;
      while (pw < T) {
        pw <<= 1;
        ++lp;
      }
      for (int32_t x = T + lane; x < pw; x += 32) {
        pcol[x] = INT32_MAX;
        pval[x] = V(0);
      }
      __syncwarp();
      for (int ls = 1; ls <= lp; ++ls)
        for (int lj = ls - 1; lj >= 0; --lj) {
          const int size = 1 << ls, j = 1 << lj;
          for (int t = lane; t < (pw >> 1); t += 32) {
            const int hi = t >> lj, lo = t & (j - 1);
            int x, y;
            if (lj == ls - 1) {
              x = hi * size + lo;
              y = hi * size + size - 1 - lo;
            } else {
              x = (hi << (lj + 1)) + lo;
              y = x + j;
            }
            const int32_t kx = pcol[x], ky = pcol[y];
            if (kx > ky) {
              const V vx = pval[x], vy = pval[y];
              pcol[x] = ky;
              pcol[y] = kx;
              pval[x] = vy;
              pval[y] = vx;
            }
          }
          __syncwarp();
        }
      int32_t carry_key = INT32_MIN;
      V carry = V(0);
      for (int32_t base = 0; base < T; base += 32) {
        const int32_t x = base + lane;
        const int32_t kc = x < T ? pcol[x] : INT32_MAX;
        const V kv = x < T ? pval[x] : V(0);
        const int32_t next = x + 1 < T ? pcol[x + 1] : INT32_MAX;
        V run = kv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const V y = __shfl_up_sync(0xffffffffu, run, d);
          const int32_t cy = __shfl_up_sync(0xffffffffu, kc, d);
          if (lane >= d && cy == kc) run += y;
        }
        if (kc == carry_key) run += carry;  // the run began in an earlier window
        const bool last = x < T && next != kc;
        const unsigned lm = __ballot_sync(0xffffffffu, last);
        carry_key = __shfl_sync(0xffffffffu, kc, 31);
        carry = __shfl_sync(0xffffffffu, run, 31);
        __syncwarp();
        if (last) {
          const int32_t t = r + __popc(lm & ((1u << lane) - 1u));
          pcol[t] = kc;
          pval[t] = run;
        }
        r += __popc(lm);
        __syncwarp();
      }
    }
    __syncwarp();
    // (3) the pI x r terms of the outer product, spread over the lanes
    //     (pair e = s * r + t; one division a row, then steps of 32 pairs)
    if (r > 0) {
      const int32_t q = 32 / r, rem = 32 - q * r;
      int32_t s = lane / r, t = lane - s * r;
      for (int32_t e = lane; e < pI * r; e += 32) {
        const int32_t i = wi[s];
        if (i >= i0 && i < i1)
          add_term(acc, col, sm.roff[i - i0], sm.roff[i - i0 + 1], pcol[t], ww[s] * pval[t], on_chip, a.status);
        s += q;
        t += rem;
        if (t >= r) {
          t -= r;
          ++s;
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  if (on_chip)
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) a.c_val[base + t] = sm.acc[t];
  __syncthreads();
}

template <typename V>
__global__ void __launch_bounds__(256) k_numeric_sorted(NumArgs<V> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  SortedSmem<V> sm(smraw, a.CH, a.max_rows, blockDim.x >> 5);
  for (int32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) sorted_chunk<V>(a, c, sm);
}

template <typename V>
size_t sorted_smem_bytes(int CH, int max_rows, int threads) {
  const int nwarps = threads / 32;
  size_t b = ((size_t)CH + (size_t)nwarps * (kRowMax + 32)) * sizeof(V);
  b = (b + 15) & ~size_t(15);
  b += ((size_t)CH + max_rows + 1 + (size_t)nwarps * (kRowMax + 32)) * sizeof(int32_t);
  return (b + 15) & ~size_t(15);
}

}  // namespace

template <typename V>
int prepare_sorted_t(ptap_plan* p) {
  const size_t smem = sorted_smem_bytes<V>(p->cfg.chunk_entries, std::max(p->max_chunk_rows, 1),
                                           p->cfg.block_threads);
  PTAP_TRY(grow_smem_limit((const void*)k_numeric_sorted<V>, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_numeric_sorted<V>, p->cfg.block_threads, smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  p->num_smem = smem;
  p->num_per_sm = per_sm;
  return PTAP_OK;
}

int prepare_sorted(ptap_plan* p) {
  return p->dtype == PTAP_F64 ? prepare_sorted_t<double>(p) : prepare_sorted_t<float>(p);
}

template <typename V>
int launch_sorted_t(ptap_plan* p, const NumArgs<V>& a, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(a.nchunks, (int64_t)num_sms() * p->num_per_sm);
  if (grid <= 0) return PTAP_OK;
  k_numeric_sorted<V><<<grid, p->cfg.block_threads, p->num_smem, s>>>(a);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

template int launch_sorted_t<float>(ptap_plan*, const NumArgs<float>&, cudaStream_t);
template int launch_sorted_t<double>(ptap_plan*, const NumArgs<double>&, cudaStream_t);

}  // namespace ptap
