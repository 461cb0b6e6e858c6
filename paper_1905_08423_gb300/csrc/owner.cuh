// Device building blocks of the owner-mode numeric scheme, shared by the
// single-product kernel (numeric.cu) and the batched persistent kernel
// (batch.cu).  See numeric.cu for the scheme.
#pragma once

#include "common.cuh"

namespace ptap {

template <typename V>
struct NumArgs {
  CsrV<V> A, P;
  const int32_t* c_rp;
  const int32_t* c_ci;
  V* c_val;
  const int32_t* chunk_row;
  const int32_t* chunk_fptr;
  const int32_t* chunk_frows;
  int32_t nchunks;
  int32_t CH;        // on-chip accumulator capacity (entries)
  int32_t max_rows;  // max coarse rows per chunk
  int32_t* status;
};

// key -> slot in a power-of-two open-addressing map; -1 when full.
__device__ __forceinline__ int map_slot(int32_t* keys, int log2, int32_t j) {
  const uint32_t mask = (1u << log2) - 1u;
  uint32_t h = hash32((uint32_t)j) >> (32 - log2);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t cur = ((volatile int32_t*)keys)[h];
    if (cur == j) return (int)h;
    if (cur == kEmpty) {
      const int32_t old = atomicCAS(&keys[h], kEmpty, j);
      if (old == kEmpty || old == j) return (int)h;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

// Position of column j in the sorted segment col[lo, hi); -1 if absent.
__device__ __forceinline__ int32_t find_col(const int32_t* col, int32_t lo, int32_t hi, int32_t j) {
  const int32_t end = hi;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (col[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  return (lo < end && col[lo] == j) ? lo : -1;
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if (G == 32) return 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
}

// Adds w * v to the accumulator entry of C(i, j), i in [i0, i1).
template <typename V>
__device__ __forceinline__ void owner_add(V* acc, const int32_t* col, const int32_t* roff, int32_t i0,
                                          int32_t i, int32_t j, V wv, int32_t* status) {
  const int32_t r = i - i0;
  const int32_t pos = find_col(col, roff[r], roff[r + 1], j);
  if (pos >= 0) atomicAdd(&acc[pos], wv);
  else atomicExch(status, PTAP_ERR_PATTERN);
}

// Shared-memory carve-up of one owner-mode CTA.
template <typename V>
struct OwnerSmem {
  V* acc;
  V* hvals;
  int32_t* ccol;
  int32_t* roff;
  int32_t* hkeys;
  __device__ OwnerSmem(unsigned char* raw, int CH, int max_rows, int ngroups, int slots) {
    acc = (V*)raw;
    hvals = acc + CH;
    ccol = (int32_t*)(hvals + ngroups * slots);
    roff = ccol + CH;
    hkeys = roff + max_rows + 1;
  }
};

// One chunk of coarse rows [chunk_row[c], chunk_row[c+1]) owned by this CTA:
// zero the accumulator, visit the chunk's fine rows, form each row of A P in
// a group's hash map (Alg. 3), add P(I,i) (A P)(I,:) for the chunk's i
// (Alg. 8), write the chunk's values once.  Heavy chunks (one C row longer
// than the on-chip capacity) accumulate in C itself with atomics.
template <typename V, int G>
__device__ void owner_chunk(const NumArgs<V>& a, int32_t c, OwnerSmem<V>& sm, int32_t* gflag,
                            int slots_log2) {
  const int CH = a.CH;
  const int slots = 1 << slots_log2;
  const int group = threadIdx.x / G, glane = threadIdx.x % G, ngroups = blockDim.x / G;
  const unsigned gmask = group_mask<G>();
  int32_t* hk = sm.hkeys + group * slots;
  V* hv = sm.hvals + group * slots;
  V* acc_s = sm.acc;
  int32_t* ccol = sm.ccol;
  int32_t* roff = sm.roff;
  const int32_t i0 = a.chunk_row[c], i1 = a.chunk_row[c + 1];
  const int32_t base = a.c_rp[i0];
  const int32_t nnz = a.c_rp[i1] - base;
  const bool heavy = nnz > CH;
  V* acc = heavy ? a.c_val + base : acc_s;
  const int32_t* col = heavy ? a.c_ci + base : ccol;
  if (!heavy) {
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) {
      acc_s[t] = V(0);
      ccol[t] = a.c_ci[base + t];
    }
  } else {
    for (int64_t t = threadIdx.x; t < nnz; t += blockDim.x) acc[t] = V(0);
  }
  for (int r = threadIdx.x; r <= i1 - i0; r += blockDim.x) roff[r] = a.c_rp[i0 + r] - base;
  __syncthreads();

  const int32_t f1 = a.chunk_fptr[c + 1];
  for (int32_t f = a.chunk_fptr[c] + group; f < f1; f += ngroups) {
    const int32_t I = a.chunk_frows[f];
    for (int s = glane; s < slots; s += G) {
      hk[s] = kEmpty;
      hv[s] = V(0);
    }
    if (glane == 0) gflag[group] = 0;
    __syncwarp(gmask);
    const int32_t a0 = a.A.rp[I], a1 = a.A.rp[I + 1];
    // R = A(I,:) P  (Alg. 3)
    for (int32_t x = a0 + glane; x < a1; x += G) {
      const int32_t k = a.A.ci[x];
      const V av = a.A.val[x];
      const int32_t b1 = a.P.rp[k + 1];
      for (int32_t b = a.P.rp[k]; b < b1; ++b) {
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
    const int32_t p0 = a.P.rp[I], p1 = a.P.rp[I + 1];
    if (!((volatile int32_t*)gflag)[group]) {
      // C(i,:) += P(I,i) R  for i in P(I,:) inside the chunk  (Alg. 8)
      for (int s = glane; s < slots; s += G) {
        const int32_t j = hk[s];
        if (j == kEmpty) continue;
        const V v = hv[s];
        for (int32_t e = p0; e < p1; ++e) {
          const int32_t i = a.P.ci[e];
          if (i < i0) continue;
          if (i >= i1) break;
          owner_add(acc, col, roff, i0, i, j, a.P.val[e] * v, a.status);
        }
      }
    } else {
      // table overflow: add every product A(I,k) P(k,j) P(I,i) directly
      for (int32_t x = a0 + glane; x < a1; x += G) {
        const int32_t k = a.A.ci[x];
        const V av = a.A.val[x];
        for (int32_t b = a.P.rp[k]; b < a.P.rp[k + 1]; ++b) {
          const int32_t j = a.P.ci[b];
          const V t = av * a.P.val[b];
          for (int32_t e = p0; e < p1; ++e) {
            const int32_t i = a.P.ci[e];
            if (i < i0) continue;
            if (i >= i1) break;
            owner_add(acc, col, roff, i0, i, j, a.P.val[e] * t, a.status);
          }
        }
      }
    }
    __syncwarp(gmask);
  }
  __syncthreads();
  if (!heavy)
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) a.c_val[base + t] = acc_s[t];
  __syncthreads();
}

}  // namespace ptap
