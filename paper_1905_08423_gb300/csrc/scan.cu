// Device prefix sums and segmented sorts used by the symbolic phases.
//
// The symbolic phase of the paper turns per-row counts into the preallocated
// storage of C (Section 2, Alg. 2: "preallocate memory using nzd and nzo";
// Section 3, Alg. 7).  On the GPU that is an exclusive scan of the row counts
// into row_ptr, with the total checked against the int32 index range.
#include "common.cuh"

namespace ptap {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  T off = w ? warp_sums[w - 1] : T(0);
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return off + x - v;
}

// Sum of each tile of kScanTile input elements.
template <typename T>
__global__ void k_tile_sums(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += (int64_t)in[base + k];
  int64_t tot;
  block_exclusive_scan<int64_t>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of one tile; adds tile_off[tile] (or 0); writes out[i] for
// i < n, and out[n] = grand total when this tile holds the last element.
template <typename TI, typename TO>
__global__ void k_scan_tiles(const TI* __restrict__ in, int64_t n, const int64_t* __restrict__ tile_off,
                             TO* __restrict__ out, int64_t grand_total_index) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? (int64_t)in[base + k] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t pre = block_exclusive_scan<int64_t>(s, &tot);
  const int64_t off = tile_off ? tile_off[blockIdx.x] : 0;
  pre += off;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = (TO)pre;
    pre += v[k];
  }
  const int64_t last_tile = n > 0 ? (n - 1) / kScanTile : 0;
  if (grand_total_index >= 0 && blockIdx.x == last_tile && threadIdx.x == 0)
    out[grand_total_index] = (TO)(off + tot);
}

}  // namespace

// Exclusive scan of int64 a[0..n) in place, with a[n] = total.
static int scan_i64_inplace(Tracker& mem, int64_t* a, int64_t n, cudaStream_t s) {
  const int64_t tiles = ceil_div(n > 0 ? n : 1, kScanTile);
  if (tiles == 1) {
    k_scan_tiles<int64_t, int64_t><<<1, kScanThreads, 0, s>>>(a, n, nullptr, a, n);
    PTAP_LAUNCHED();
    return PTAP_OK;
  }
  Scratch sc(&mem);
  int64_t* sums = nullptr;
  PTAP_TRY(sc.get(&sums, tiles + 1));
  k_tile_sums<int64_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(a, n, sums);
  PTAP_LAUNCHED();
  PTAP_TRY(scan_i64_inplace(mem, sums, tiles, s));
  k_scan_tiles<int64_t, int64_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(a, n, sums, a, n);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

int exclusive_scan(Tracker& mem, const int32_t* in, int32_t* out, int64_t n, int64_t* total,
                   cudaStream_t s) {
  const int64_t tiles = ceil_div(n > 0 ? n : 1, kScanTile);
  Scratch sc(&mem);
  int64_t* sums = nullptr;
  PTAP_TRY(sc.get(&sums, tiles + 1));
  k_tile_sums<int32_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  PTAP_LAUNCHED();
  PTAP_TRY(scan_i64_inplace(mem, sums, tiles, s));
  int64_t h_total = 0;
  PTAP_CUDA(cudaMemcpyAsync(&h_total, sums + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  if (h_total >= ((int64_t)1 << 31)) return PTAP_ERR_OVERFLOW;
  k_scan_tiles<int32_t, int32_t><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out, n);
  PTAP_LAUNCHED();
  if (n == 0) PTAP_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
  if (total) *total = h_total;
  return PTAP_OK;
}

// ---------------------------------------------------------------------------
// segmented sort
//
// Bitonic network in the form where every comparator puts the smaller key at
// the lower index: merge stage k first compares i with its mirror inside the
// k-block, then i with i ^ j for j = k/4 .. 1.  Missing elements past the
// segment end act as +infinity and never move, so segments need no padding.
// ---------------------------------------------------------------------------
namespace {

constexpr int kSortSmem = 4096;

__device__ __forceinline__ void cmp_swap(int32_t* k, int32_t* v, int a, int b) {
  int32_t ka = k[a], kb = k[b];
  if (ka > kb) {
    k[a] = kb;
    k[b] = ka;
    if (v) {
      int32_t t = v[a];
      v[a] = v[b];
      v[b] = t;
    }
  }
}

// Warp per segment of length <= 32: registers and shuffles.
__global__ void k_sort_warp(const int32_t* __restrict__ ptr, int32_t nseg, int32_t* keys,
                            int32_t* vals) {
  const int lane = threadIdx.x & 31;
  const int64_t seg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (seg >= nseg) return;
  const int32_t b = ptr[seg], e = ptr[seg + 1], len = e - b;
  if (len <= 1 || len > 32) return;
  int32_t k = lane < len ? keys[b + lane] : INT32_MAX;
  int32_t v = (vals && lane < len) ? vals[b + lane] : 0;
  for (int size = 2; size <= 32; size <<= 1) {
    for (int j = size >> 1; j > 0; j >>= 1) {
      const int partner = (j == (size >> 1)) ? (lane ^ (size - 1)) : (lane ^ j);
      const int32_t pk = __shfl_sync(0xffffffffu, k, partner);
      const int32_t pv = __shfl_sync(0xffffffffu, v, partner);
      const bool lower = lane < partner;
      const bool take = lower ? (pk < k) : (pk > k);
      if (take) {
        k = pk;
        v = pv;
      }
    }
  }
  if (lane < len) {
    keys[b + lane] = k;
    if (vals) vals[b + lane] = v;
  }
}

// Bitonic over n elements of k/v (shared or global), by a whole CTA.
__device__ void cta_bitonic(int32_t* k, int32_t* v, int n) {
  int p = 1;
  while (p < n) p <<= 1;
  for (int size = 2; size <= p; size <<= 1) {
    for (int j = size >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (p >> 1); t += blockDim.x) {
        int a, b;
        if (j == (size >> 1)) {
          const int blk = t / j, off = t % j;
          a = blk * size + off;
          b = blk * size + size - 1 - off;
        } else {
          a = (t / j) * 2 * j + (t % j);
          b = a + j;
        }
        if (b < n) cmp_swap(k, v, a, b);
      }
      __syncthreads();
    }
  }
}

// A CTA per listed segment: segments of at most `cap` elements are sorted in
// dynamic shared memory (cap keys, then cap values when vals is set), longer
// ones in place in global memory.
__global__ void k_sort_cta_list(const int32_t* __restrict__ ptr, const int32_t* __restrict__ list,
                                int32_t nlist, int32_t* keys, int32_t* vals, int32_t cap) {
  extern __shared__ int32_t sort_smem[];
  int32_t* sk = sort_smem;
  int32_t* sv = sort_smem + cap;
  for (int32_t li = blockIdx.x; li < nlist; li += gridDim.x) {
    const int32_t seg = list[li];
    const int32_t b = ptr[seg], len = ptr[seg + 1] - b;
    if (len <= cap) {
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        sk[t] = keys[b + t];
        if (vals) sv[t] = vals[b + t];
      }
      __syncthreads();
      cta_bitonic(sk, vals ? sv : nullptr, len);
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        keys[b + t] = sk[t];
        if (vals) vals[b + t] = sv[t];
      }
    } else {
      cta_bitonic(keys + b, vals ? vals + b : nullptr, len);
    }
    __syncthreads();
  }
}

// Segments longer than 32 into list; count[0] their number, count[1] the
// longest length.
__global__ void k_list_long(const int32_t* __restrict__ ptr, int32_t nseg, int32_t* list,
                            int32_t* count) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int32_t len = ptr[s + 1] - ptr[s];
  if (len > 32) {
    list[atomicAdd(&count[0], 1)] = (int32_t)s;
    atomicMax(&count[1], len);
  }
}

}  // namespace

int segmented_sort(Tracker& mem, const int32_t* ptr, int32_t nseg, int32_t* keys, int32_t* vals,
                   int32_t max_len, cudaStream_t s) {
  if (nseg <= 0) return PTAP_OK;
  {
    const int64_t threads = (int64_t)nseg * 32;
    k_sort_warp<<<(unsigned)ceil_div(threads, 256), 256, 0, s>>>(ptr, nseg, keys, vals);
    PTAP_LAUNCHED();
  }
  if (max_len >= 0 && max_len <= 32) return PTAP_OK;
  Scratch sc(&mem);
  int32_t *list = nullptr, *cnt = nullptr;
  PTAP_TRY(sc.get(&list, nseg));
  PTAP_TRY(sc.get(&cnt, 2));
  PTAP_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(int32_t), s));
  k_list_long<<<(unsigned)ceil_div(nseg, 256), 256, 0, s>>>(ptr, nseg, list, cnt);
  PTAP_LAUNCHED();
  int32_t h[2] = {0, 0};
  PTAP_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  if (h[0] > 0) {
    // the shared-memory tile grows to the longest segment, up to the
    // device's opt-in limit; long tiles get 1024-thread CTAs
    const int eb = vals ? 8 : 4;
    int32_t cap = kSortSmem;
    if (h[1] > kSortSmem) {
      int dev = 0, optin = 0;
      PTAP_CUDA(cudaGetDevice(&dev));
      PTAP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      cap = std::max<int32_t>(kSortSmem, std::min<int64_t>(h[1], optin / eb));
    }
    const size_t bytes = (size_t)cap * eb;
    static size_t attr = 48 * 1024;  // largest dynamic size set so far (the default allows 48 KB)
    if (bytes > attr) {
      PTAP_TRY(grow_smem_limit((const void*)k_sort_cta_list, (int)bytes));
      attr = bytes;
    }
    const bool big = cap > kSortSmem;
    const int grid = (int)std::min<int64_t>(h[0], (int64_t)num_sms() * (big ? 1 : 8));
    k_sort_cta_list<<<grid, big ? 1024 : 256, bytes, s>>>(ptr, list, h[0], keys, vals, cap);
    PTAP_LAUNCHED();
  }
  return PTAP_OK;
}

}  // namespace ptap
