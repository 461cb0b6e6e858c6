// Batched numeric products: many triple products of uneven sizes (every level
// of a hierarchy, or independent systems) in one persistent launch.
//
// Each problem keeps its own plan (symbolic phase reused, Section 4.1's "one
// symbolic, many numeric"; Section 4.2's caching of intermediate data).  The
// batch flattens every problem's owner-mode chunks into one work queue sorted
// by estimated work (fine rows visited), longest first, and launches one CTA
// per SM slot; each CTA pops items with an atomic counter until the queue is
// empty.  There is no wait on another CTA anywhere.  The launch reads only
// device pointers fixed at creation, so a CUDA graph that captures it stays
// valid while the caller rewrites the values of A and P in place.
#include <algorithm>
#include <new>
#include <numeric>

#include "fastkern.cuh"
#include "owner.cuh"

namespace ptap {

size_t owner_smem_for(int dtype, const Config& c, int max_rows);

template <typename V, int G>
__global__ void __launch_bounds__(256) k_batch_owner(const NumArgs<V>* __restrict__ probs,
                                                    const int32_t* __restrict__ items, int32_t nitems,
                                                    int32_t* counter, int slots_log2, int CH,
                                                    int max_rows) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t gflag[256 / 4];
  __shared__ int32_t item;
  OwnerSmem<V> sm(smraw, CH, max_rows, blockDim.x / G, 1 << slots_log2);
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t it = item;
    __syncthreads();
    if (it >= nitems) break;
    const int32_t prob = items[2 * it], chunk = items[2 * it + 1];
    const NumArgs<V> a = probs[prob];
    owner_chunk<V, G>(a, chunk, sm, gflag, slots_log2);
  }
}

// Fast variant: every plan of the batch runs class programs (interpreted).
struct NoSpecial {
  template <typename V>
  __device__ bool operator()(const ptapk::FastArgs<V>&, int32_t, int32_t, int32_t, int32_t, int32_t, V*,
                             const int32_t*, int32_t) const {
    return false;
  }
};

template <typename V>
__global__ void __launch_bounds__(256) k_batch_fast(const ptapk::FastArgs<V>* __restrict__ probs,
                                                   const int32_t* __restrict__ items, int32_t nitems,
                                                   int32_t* counter, int CH, int maxr, int max_rows,
                                                   int prog_cap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t item;
  ptapk::FastSmem<V> sm(smraw, CH, maxr, max_rows, prog_cap);
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t it = item;
    __syncthreads();
    if (it >= nitems) break;
    const ptapk::FastArgs<V> a = probs[items[2 * it]];
    ptapk::fast_chunk<V>(a, items[2 * it + 1], sm, NoSpecial());
  }
}

template <typename V>
static int batch_create_t(ptap_batch* b, ptap_plan* const* plans, const ptap_csr* A,
                          const ptap_csr* P, void* const* C, cudaStream_t s) {
  std::vector<NumArgs<V>> h(b->count);
  std::vector<ptapk::FastArgs<V>> hf(b->count);
  std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>> work;
  for (int32_t q = 0; q < b->count; ++q) {
    ptap_plan* p = plans[q];
    if (b->fast) {
      ptapk::FastArgs<V>& f = hf[q];
      f.A = ptapk::FCsr<V>{A[q].nrows, A[q].ncols, A[q].row_ptr, A[q].col_idx, (const V*)A[q].val};
      f.P = ptapk::FCsr<V>{P[q].nrows, P[q].ncols, P[q].row_ptr, P[q].col_idx, (const V*)P[q].val};
      f.c_rp = p->c_rp;
      f.c_val = (V*)C[q];
      f.chunk_row = p->chunk_row;
      f.chunk_piece = p->chunk_piece;
      f.piece_f0 = p->piece_f0;
      f.piece_meta = p->piece_meta;
      f.frows = p->chunk_frows;
      f.pool = p->class_pool;
      f.class_off = p->class_off;
      f.nchunks = p->nchunks;
      f.CH = p->cfg.chunk_entries;
      f.max_rows = std::max(p->max_chunk_rows, 1);
      f.prog_cap = (p->class_maxlen + 15) & ~15;
      f.maxr = std::max(p->class_maxr, 1);
      f.work = nullptr;  // the batch has its own queue
      f.chunk_order = nullptr;
      f.rs_global = nullptr;
      f.jit_slot = nullptr;
      f.aq = p->aq;
      f.crows = p->compact ? p->chunk_crows : nullptr;
      f.row_loc = p->compact ? p->row_loc : nullptr;
      f.chunk_nnz = p->compact ? p->chunk_nnz : nullptr;
      f.loc_bits = p->loc_bits;
    }
    NumArgs<V>& a = h[q];
    a.A = CsrV<V>{A[q].nrows, A[q].ncols, A[q].row_ptr, A[q].col_idx, (const V*)A[q].val};
    a.P = CsrV<V>{P[q].nrows, P[q].ncols, P[q].row_ptr, P[q].col_idx, (const V*)P[q].val};
    a.c_rp = p->c_rp;
    a.c_ci = p->c_ci;
    a.c_val = (V*)C[q];
    a.chunk_row = p->chunk_row;
    a.chunk_fptr = p->chunk_fptr;
    a.chunk_frows = p->chunk_frows;
    a.nchunks = p->nchunks;
    a.CH = p->cfg.chunk_entries;
    a.max_rows = b->max_chunk_rows;
    a.status = b->status;
    std::vector<int32_t> fptr(p->nchunks + 1);
    PTAP_CUDA(cudaMemcpyAsync(fptr.data(), p->chunk_fptr, fptr.size() * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, s));
    PTAP_CUDA(cudaStreamSynchronize(s));
    for (int32_t c = 0; c < p->nchunks; ++c)
      work.push_back({(int64_t)fptr[c + 1] - fptr[c], {q, c}});
  }
  std::stable_sort(work.begin(), work.end(),
                   [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<int32_t> items(2 * work.size() + 2, 0);
  for (size_t t = 0; t < work.size(); ++t) {
    items[2 * t] = work[t].second.first;
    items[2 * t + 1] = work[t].second.second;
  }
  b->total_items = (int64_t)work.size();
  const size_t dbytes = b->fast ? hf.size() * sizeof(ptapk::FastArgs<V>) : h.size() * sizeof(NumArgs<V>);
  PTAP_TRY(b->mem.get(&b->d_desc, dbytes));
  PTAP_TRY(b->mem.get_n(&b->d_items, (int64_t)items.size()));
  if (b->fast)
    PTAP_CUDA(cudaMemcpyAsync(b->d_desc, hf.data(), dbytes, cudaMemcpyHostToDevice, s));
  else
    PTAP_CUDA(cudaMemcpyAsync(b->d_desc, h.data(), dbytes, cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  return PTAP_OK;
}

template <typename V>
static int batch_prepare_fast(ptap_batch* b) {
  const size_t smem = ptapk::fast_smem_bytes<V>(b->fast_ch, b->cfg.block_threads, b->fast_maxr,
                                                b->max_chunk_rows, b->fast_prog_cap);
  PTAP_CUDA(cudaFuncSetAttribute(k_batch_fast<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_fast<V>, b->cfg.block_threads, smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  b->smem = smem;
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->total_items, (int64_t)num_sms() * per_sm));
  return PTAP_OK;
}

template <typename V>
static int batch_launch_fast(ptap_batch* b, cudaStream_t s) {
  PTAP_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), s));
  k_batch_fast<V><<<b->grid, b->cfg.block_threads, b->smem, s>>>(
      (const ptapk::FastArgs<V>*)b->d_desc, b->d_items, (int32_t)b->total_items, b->d_counter, b->fast_ch,
      b->fast_maxr, b->max_chunk_rows, b->fast_prog_cap);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

template <typename V, int G>
static int batch_prepare_g(ptap_batch* b) {
  const Config& c = b->cfg;
  const size_t smem = owner_smem_for(b->dtype, c, b->max_chunk_rows);
  PTAP_CUDA(cudaFuncSetAttribute(k_batch_owner<V, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_owner<V, G>, c.block_threads,
                                                          smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  b->smem = smem;
  b->grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->total_items, (int64_t)num_sms() * per_sm));
  return PTAP_OK;
}

template <typename V, int G>
static int batch_launch_g(ptap_batch* b, cudaStream_t s) {
  const Config& c = b->cfg;
  const int slots_log2 = c.force_spill ? 2 : ilog2_ceil((uint32_t)std::max(4, c.ap_slots));
  PTAP_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), s));
  k_batch_owner<V, G><<<b->grid, c.block_threads, b->smem, s>>>(
      (const NumArgs<V>*)b->d_desc, b->d_items, (int32_t)b->total_items, b->d_counter, slots_log2,
      c.chunk_entries, b->max_chunk_rows);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

// Evaluates CALL with V (value type) and G (group width) bound to the batch's.
#define PTAP_BATCH_DISPATCH(b, CALL)                               \
  do {                                                             \
    const int _g = (b)->cfg.group_lanes;                           \
    if ((b)->dtype == PTAP_F64) {                                  \
      using V = double;                                            \
      if (_g == 4) { constexpr int G = 4; return CALL; }           \
      if (_g == 8) { constexpr int G = 8; return CALL; }           \
      if (_g == 16) { constexpr int G = 16; return CALL; }         \
      if (_g == 32) { constexpr int G = 32; return CALL; }         \
    } else {                                                       \
      using V = float;                                             \
      if (_g == 4) { constexpr int G = 4; return CALL; }           \
      if (_g == 8) { constexpr int G = 8; return CALL; }           \
      if (_g == 16) { constexpr int G = 16; return CALL; }         \
      if (_g == 32) { constexpr int G = 32; return CALL; }         \
    }                                                              \
    return PTAP_ERR_INVALID;                                       \
  } while (0)

static int batch_prepare(ptap_batch* b) {
  if (b->fast) return b->dtype == PTAP_F64 ? batch_prepare_fast<double>(b) : batch_prepare_fast<float>(b);
  PTAP_BATCH_DISPATCH(b, (batch_prepare_g<V, G>(b)));
}

static int batch_launch(ptap_batch* b, cudaStream_t s) {
  if (b->fast) return b->dtype == PTAP_F64 ? batch_launch_fast<double>(b, s) : batch_launch_fast<float>(b, s);
  PTAP_BATCH_DISPATCH(b, (batch_launch_g<V, G>(b, s)));
}

int check_numeric_inputs(const ptap_plan* p, const ptap_csr* A, const ptap_csr* P);

}  // namespace ptap

extern "C" int ptap_batch_create(ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P,
                                 void* const* C_vals, int32_t count, const ptap_allocator* alloc,
                                 void* stream, ptap_batch** out) {
  if (!out || count <= 0 || !plans || !A || !P || !C_vals) return PTAP_ERR_INVALID;
  *out = nullptr;
  const ptap_plan* p0 = plans[0];
  if (!p0) return PTAP_ERR_INVALID;
  int32_t max_rows = 1, fast_ch = 1, fast_maxr = 1, fast_prog_cap = 16;
  bool all_fast = true;
  for (int32_t q = 0; q < count; ++q) {
    const ptap_plan* p = plans[q];
    if (!p || p->kind != 0 || p->dtype != p0->dtype) return PTAP_ERR_INVALID;
    all_fast = all_fast && p->fast && p->cfg.mode == PTAP_MODE_OWNER;
    fast_ch = std::max(fast_ch, p->cfg.chunk_entries);
    fast_maxr = std::max(fast_maxr, p->class_maxr);
    fast_prog_cap = std::max(fast_prog_cap, (p->class_maxlen + 15) & ~15);
  }
  for (int32_t q = 0; q < count && !all_fast; ++q) {
    const ptap_plan* p = plans[q];
    if (p->compact) return PTAP_ERR_UNSUPPORTED;  // the general batch kernel takes row ranges
    if (p->cfg.chunk_entries != p0->cfg.chunk_entries || p->cfg.group_lanes != p0->cfg.group_lanes ||
        p->cfg.ap_slots != p0->cfg.ap_slots || p->cfg.block_threads != p0->cfg.block_threads ||
        p->cfg.force_spill != p0->cfg.force_spill)
      return PTAP_ERR_INVALID;
  }
  for (int32_t q = 0; q < count; ++q) {
    const ptap_plan* p = plans[q];
    PTAP_TRY(ptap::check_numeric_inputs(p, &A[q], &P[q]));
    if (p->nnz_c > 0 && !C_vals[q]) return PTAP_ERR_INVALID;
    max_rows = std::max(max_rows, p->max_chunk_rows);
  }
  cudaStream_t s = (cudaStream_t)stream;
  ptap_batch* b = new (std::nothrow) ptap_batch();
  if (!b) return PTAP_ERR_OOM;
  b->mem.init(alloc, s);
  b->dtype = p0->dtype;
  b->count = count;
  b->cfg = p0->cfg;
  b->cfg.block_threads = std::min(b->cfg.block_threads, 256);  // the batch kernels' bound
  b->max_chunk_rows = max_rows;
  b->fast = all_fast;
  b->fast_ch = fast_ch;
  b->fast_maxr = fast_maxr;
  b->fast_prog_cap = fast_prog_cap;
  int rc = b->mem.get_n(&b->d_counter, 1);
  if (rc == PTAP_OK) rc = b->mem.get_n(&b->status, 1);
  if (rc == PTAP_OK && cudaMemsetAsync(b->status, 0, sizeof(int32_t), s) != cudaSuccess) rc = PTAP_ERR_CUDA;
  if (rc == PTAP_OK)
    rc = b->dtype == PTAP_F64 ? ptap::batch_create_t<double>(b, plans, A, P, C_vals, s)
                              : ptap::batch_create_t<float>(b, plans, A, P, C_vals, s);
  if (rc == PTAP_OK) rc = ptap::batch_prepare(b);
  if (rc != PTAP_OK) {
    cudaStreamSynchronize(s);
    b->mem.release_all();
    delete b;
    return rc;
  }
  *out = b;
  return PTAP_OK;
}

extern "C" int ptap_batch_numeric(ptap_batch* b, void* stream) {
  ptap::Range range("ptap_batch_numeric");
  if (!b) return PTAP_ERR_INVALID;
  if (b->total_items == 0) return PTAP_OK;
  return ptap::batch_launch(b, (cudaStream_t)stream);
}

extern "C" void ptap_batch_destroy(ptap_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->mem.stream);
  b->mem.release_all();
  delete b;
}
