// Batched numeric products: many triple products of uneven sizes (every level
// of a hierarchy, or independent systems) in one persistent launch per kernel
// kind.
//
// Each problem keeps its own plan (symbolic phase reused, Section 4.1's "one
// symbolic, many numeric"; Section 4.2's caching of intermediate data).  The
// batch flattens every problem's owner-mode chunks into work queues sorted by
// estimated work (fine rows visited), longest first: one queue for problems
// whose plans run class programs, one for the others.  Each queue is served
// by one launch whose CTAs (at most one wave of resident CTAs) pop items with
// an atomic counter until the queue is empty; there is no wait on another CTA
// anywhere.  The class-program launch runs the batch's most visited class
// programs as code specialised for the batch (the programs of all its plans
// pooled by their bytes, compiled with NVRTC) when the plans ask for
// specialisation, and interprets the rest.  The launches read only device
// pointers fixed at creation, so a CUDA graph that captures them stays valid
// while the caller rewrites the values of A and P in place.
#include <algorithm>
#include <new>
#include <vector>

#include "fastkern.cuh"
#include "owner.cuh"

namespace ptap {

size_t owner_smem_for(int dtype, const Config& c, int max_rows);
int check_numeric_inputs(const ptap_plan* p, const ptap_csr* A, const ptap_csr* P);
int jit_prepare_batch(ptap_plan* const* plans, int count, int max_classes, int threads, Tracker& mem,
                      cudaStream_t s, void** fn, std::vector<int32_t*>& slots, int* nhot, double* coverage);
int jit_occupancy(void* fn, int threads, size_t smem, int* per_sm);
int jit_launch_raw(void* fn, void** params, int grid, int threads, size_t smem, cudaStream_t s);

namespace {

constexpr int kBatchGeneralThreads = 256;

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
    const NumArgs<V> a = probs[items[2 * it]];
    owner_chunk<V, G>(a, items[2 * it + 1], sm, gflag, slots_log2);
  }
}

struct NoSpecial {
  template <typename V>
  __device__ bool operator()(const ptapk::FastArgs<V>&, int32_t, int32_t, int32_t, int32_t, int32_t, V*,
                             const int32_t*, int32_t, const int32_t*) const {
    return false;
  }
};

// Interpreter for the class-program items (MaxT: 256, or 1024 for batches of
// plans built with large CTAs).
template <typename V, int MaxT>
__global__ void __launch_bounds__(MaxT) k_batch_fast(const ptapk::FastArgs<V>* __restrict__ probs,
                                                    const int32_t* __restrict__ items, int32_t nitems,
                                                    int32_t* counter, int CH, int maxr, int max_rows,
                                                    int prog_cap, V* rs) {
  ptapk::fast_batch_body<V>(probs, items, nitems, counter, CH, maxr, max_rows, prog_cap, rs, NoSpecial());
}

template <typename V>
auto fast_kernel(int threads) {
  return threads > 256 ? k_batch_fast<V, 1024> : k_batch_fast<V, 256>;
}

int optin_smem(const void* fn, int* out) {
  int dev = 0, optin = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  PTAP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (fn) {
    cudaFuncAttributes fa{};
    PTAP_CUDA(cudaFuncGetAttributes(&fa, fn));
    optin -= (int)fa.sharedSizeBytes;
  }
  *out = optin;
  return PTAP_OK;
}

// Work items of one plan, (work, problem, chunk) with work = fine rows visited.
int add_items(ptap_plan* p, int32_t q, cudaStream_t s, std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>>& w) {
  std::vector<int32_t> fptr(p->nchunks + 1);
  PTAP_CUDA(cudaMemcpyAsync(fptr.data(), p->chunk_fptr, fptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  for (int32_t c = 0; c < p->nchunks; ++c) w.push_back({(int64_t)fptr[c + 1] - fptr[c], {q, c}});
  return PTAP_OK;
}

int upload_items(ptap_batch* b, std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>>& w, int32_t** out,
                 cudaStream_t s) {
  std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<int32_t> items(2 * w.size() + 2, 0);
  for (size_t t = 0; t < w.size(); ++t) {
    items[2 * t] = w[t].second.first;
    items[2 * t + 1] = w[t].second.second;
  }
  PTAP_TRY(b->mem.get_n(out, (int64_t)items.size()));
  PTAP_CUDA(cudaMemcpyAsync(*out, items.data(), items.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));  // the host vector goes out of scope
  return PTAP_OK;
}

// Class-program side: descriptors, the kernel (specialised or interpreted)
// and its launch configuration.
template <typename V>
int prepare_fast_side(ptap_batch* b, const std::vector<ptap_plan*>& fp, const std::vector<int32_t>& fq,
                      ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P, void* const* C,
                      cudaStream_t s) {
  bool want_jit = false;
  int max_classes = 0;
  for (ptap_plan* p : fp) {
    b->fast_threads = std::max(b->fast_threads, p->cfg.block_threads);
    b->fast_ch = std::max(b->fast_ch, p->cfg.chunk_entries);
    b->fast_maxr = std::max(b->fast_maxr, p->class_maxr);
    b->fast_prog_cap = std::max(b->fast_prog_cap, (p->class_maxlen + 15) & ~15);
    b->fast_max_rows = std::max(b->fast_max_rows, p->max_chunk_rows);
    want_jit = want_jit || p->cfg.jit;
    max_classes = std::max(max_classes, p->cfg.jit ? p->cfg.jit_max_classes : 0);
  }
  std::vector<int32_t*> slots;
  if (want_jit &&
      jit_prepare_batch(fp.data(), (int)fp.size(), max_classes, b->fast_threads, b->mem, s, &b->jit_fn, slots,
                        &b->jit_classes, &b->jit_coverage) != PTAP_OK)
    b->jit_fn = nullptr;  // the interpreter serves the batch
  const size_t vb = sizeof(V);
  int per_sm = 0;
  bool rs_global = true;
  if (b->jit_fn) {
    b->fast_smem = ptapk::fast_smem_bytes<V>(b->fast_ch, b->fast_threads, b->fast_maxr, b->fast_max_rows,
                                             b->fast_prog_cap, false);
    if (jit_occupancy(b->jit_fn, b->fast_threads, b->fast_smem, &per_sm) != PTAP_OK) b->jit_fn = nullptr;
  }
  if (!b->jit_fn) {
    auto k = fast_kernel<V>(b->fast_threads);
    int optin = 0;
    PTAP_TRY(optin_smem((const void*)k, &optin));
    for (int in_smem = 1; in_smem >= 0 && per_sm < 1; --in_smem) {
      const size_t smem = ptapk::fast_smem_bytes<V>(b->fast_ch, b->fast_threads, b->fast_maxr, b->fast_max_rows,
                                                    b->fast_prog_cap, in_smem != 0);
      if (smem > (size_t)optin) continue;
      PTAP_TRY(grow_smem_limit((const void*)k, (int)smem));
      PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, b->fast_threads, smem));
      b->fast_smem = smem;
      rs_global = in_smem == 0;
    }
    if (per_sm < 1) return PTAP_ERR_UNSUPPORTED;
  }
  b->fast_grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->n_fast, (int64_t)num_sms() * per_sm));
  if (rs_global)
    PTAP_TRY(b->mem.get(&b->fast_rs, (size_t)b->fast_grid * b->fast_threads * b->fast_maxr * vb));
  std::vector<ptapk::FastArgs<V>> hf(b->count);
  for (size_t i = 0; i < fp.size(); ++i) {
    const int32_t q = fq[i];
    ptap_plan* p = plans[q];
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
    f.jit_slot = b->jit_fn ? slots[i] : nullptr;
    f.aq = p->aq;
    f.rec = p->rec;
    f.rec_off = p->rec_off;
    f.crows = p->compact ? p->chunk_crows : nullptr;
    f.row_loc = p->compact ? p->row_loc : nullptr;
    f.chunk_nnz = p->compact ? p->chunk_nnz : nullptr;
    f.loc_bits = p->loc_bits;
  }
  PTAP_TRY(b->mem.get(&b->d_desc_fast, hf.size() * sizeof(ptapk::FastArgs<V>)));
  PTAP_CUDA(cudaMemcpyAsync(b->d_desc_fast, hf.data(), hf.size() * sizeof(ptapk::FastArgs<V>),
                            cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  return PTAP_OK;
}

// General side: descriptors and the owner-mode kernel's launch configuration.
// Its on-chip capacity is the largest chunk of the general plans, lowered to
// what a CTA's shared memory holds; a chunk above it accumulates in C with
// atomics (the kernel's heavy path).
template <typename V, int G>
int prepare_gen_side(ptap_batch* b, const std::vector<int32_t>& gq, ptap_plan* const* plans,
                     const ptap_csr* A, const ptap_csr* P, void* const* C, cudaStream_t s) {
  Config& c = b->cfg;
  c.block_threads = kBatchGeneralThreads;
  int optin = 0;
  PTAP_TRY(optin_smem((const void*)k_batch_owner<V, G>, &optin));
  Config c0 = c;
  c0.chunk_entries = 0;
  const size_t fixed = owner_smem_for(b->dtype, c0, b->max_chunk_rows);
  if (fixed + 64 * (sizeof(V) + sizeof(int32_t)) > (size_t)optin) return PTAP_ERR_UNSUPPORTED;
  const int64_t fit = ((int64_t)optin - (int64_t)fixed) / (int64_t)(sizeof(V) + sizeof(int32_t));
  c.chunk_entries = (int)std::max<int64_t>(64, std::min<int64_t>(c.chunk_entries, fit & ~int64_t(63)));
  b->gen_smem = owner_smem_for(b->dtype, c, b->max_chunk_rows);
  PTAP_TRY(grow_smem_limit((const void*)k_batch_owner<V, G>, (int)b->gen_smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_owner<V, G>, c.block_threads,
                                                          b->gen_smem));
  if (per_sm < 1) return PTAP_ERR_UNSUPPORTED;
  b->gen_grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->n_gen, (int64_t)num_sms() * per_sm));
  std::vector<NumArgs<V>> h(b->count);
  for (int32_t q : gq) {
    ptap_plan* p = plans[q];
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
    a.CH = std::min(p->cfg.chunk_entries, c.chunk_entries);
    a.max_rows = b->max_chunk_rows;
    a.status = b->status;
  }
  PTAP_TRY(b->mem.get(&b->d_desc_gen, h.size() * sizeof(NumArgs<V>)));
  PTAP_CUDA(cudaMemcpyAsync(b->d_desc_gen, h.data(), h.size() * sizeof(NumArgs<V>), cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  return PTAP_OK;
}

template <typename V, int G>
int launch_t(ptap_batch* b, cudaStream_t s) {
  PTAP_CUDA(cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(int32_t), s));
  if (b->n_fast > 0) {
    const ptapk::FastArgs<V>* probs = (const ptapk::FastArgs<V>*)b->d_desc_fast;
    int32_t nitems = (int32_t)b->n_fast;
    V* rs = (V*)b->fast_rs;
    if (b->jit_fn) {
      int32_t* counter = b->d_counter;
      const int32_t* items = b->d_items_fast;
      void* params[] = {(void*)&probs, (void*)&items, (void*)&nitems, (void*)&counter, (void*)&b->fast_ch,
                        (void*)&b->fast_maxr, (void*)&b->fast_max_rows, (void*)&b->fast_prog_cap, (void*)&rs};
      PTAP_TRY(jit_launch_raw(b->jit_fn, params, b->fast_grid, b->fast_threads, b->fast_smem, s));
    } else {
      fast_kernel<V>(b->fast_threads)<<<b->fast_grid, b->fast_threads, b->fast_smem, s>>>(
          probs, b->d_items_fast, nitems, b->d_counter, b->fast_ch, b->fast_maxr, b->fast_max_rows,
          b->fast_prog_cap, rs);
      PTAP_LAUNCHED();
    }
  }
  if (b->n_gen > 0) {
    const Config& c = b->cfg;
    const int slots_log2 = c.force_spill ? 2 : ilog2_ceil((uint32_t)std::max(4, c.ap_slots));
    k_batch_owner<V, G><<<b->gen_grid, c.block_threads, b->gen_smem, s>>>(
        (const NumArgs<V>*)b->d_desc_gen, b->d_items_gen, (int32_t)b->n_gen, b->d_counter + 1, slots_log2,
        c.chunk_entries, b->max_chunk_rows);
    PTAP_LAUNCHED();
  }
  return PTAP_OK;
}

template <typename V, int G>
int create_t(ptap_batch* b, ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P, void* const* C,
             cudaStream_t s) {
  std::vector<ptap_plan*> fp;
  std::vector<int32_t> fq, gq;
  std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>> wf, wg;
  for (int32_t q = 0; q < b->count; ++q) {
    ptap_plan* p = plans[q];
    if (p->fast && p->cfg.mode == PTAP_MODE_OWNER) {
      fp.push_back(p);
      fq.push_back(q);
      PTAP_TRY(add_items(p, q, s, wf));
    } else {
      gq.push_back(q);
      PTAP_TRY(add_items(p, q, s, wg));
    }
  }
  b->n_fast = (int64_t)wf.size();
  b->n_gen = (int64_t)wg.size();
  PTAP_TRY(upload_items(b, wf, &b->d_items_fast, s));
  PTAP_TRY(upload_items(b, wg, &b->d_items_gen, s));
  if (!fp.empty()) PTAP_TRY(prepare_fast_side<V>(b, fp, fq, plans, A, P, C, s));
  if (!gq.empty()) PTAP_TRY((prepare_gen_side<V, G>(b, gq, plans, A, P, C, s)));
  return PTAP_OK;
}

// Evaluates CALL with V (value type) and G (lanes per fine row of the general
// kernel) bound to the batch's.
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

int batch_create(ptap_batch* b, ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P, void* const* C,
                 cudaStream_t s) {
  PTAP_BATCH_DISPATCH(b, (create_t<V, G>(b, plans, A, P, C, s)));
}

int batch_launch(ptap_batch* b, cudaStream_t s) { PTAP_BATCH_DISPATCH(b, (launch_t<V, G>(b, s))); }

}  // namespace

}  // namespace ptap

extern "C" int ptap_batch_create(ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P,
                                 void* const* C_vals, int32_t count, const ptap_allocator* alloc,
                                 void* stream, ptap_batch** out) {
  ptap::Range range("ptap_batch_create");
  if (!out || count <= 0 || !plans || !A || !P || !C_vals) return PTAP_ERR_INVALID;
  *out = nullptr;
  const ptap_plan* p0 = plans[0];
  if (!p0) return PTAP_ERR_INVALID;
  const ptap_plan* g0 = nullptr;  // first plan on the general kernel
  int32_t max_rows = 1, gen_ch = 64;
  for (int32_t q = 0; q < count; ++q) {
    const ptap_plan* p = plans[q];
    if (!p || p->kind != 0 || p->dtype != p0->dtype) return PTAP_ERR_INVALID;
    PTAP_TRY(ptap::check_numeric_inputs(p, &A[q], &P[q]));
    if (p->nnz_c > 0 && !C_vals[q]) return PTAP_ERR_INVALID;
    if (p->fast && p->cfg.mode == PTAP_MODE_OWNER) continue;
    // the general kernel takes row ranges, with lanes per fine row and hash
    // slots compiled in: its plans must agree on those
    if (p->compact) return PTAP_ERR_UNSUPPORTED;
    if (!g0) g0 = p;
    if (p->cfg.group_lanes != g0->cfg.group_lanes || p->cfg.ap_slots != g0->cfg.ap_slots ||
        p->cfg.force_spill != g0->cfg.force_spill)
      return PTAP_ERR_INVALID;
    gen_ch = std::max(gen_ch, p->cfg.chunk_entries);
    max_rows = std::max(max_rows, p->max_chunk_rows);
  }
  cudaStream_t s = (cudaStream_t)stream;
  ptap_batch* b = new (std::nothrow) ptap_batch();
  if (!b) return PTAP_ERR_OOM;
  b->mem.init(alloc, s);
  b->dtype = p0->dtype;
  b->count = count;
  b->cfg = g0 ? g0->cfg : p0->cfg;
  b->cfg.chunk_entries = gen_ch;
  b->max_chunk_rows = max_rows;
  int rc = b->mem.get_n(&b->d_counter, 2);
  if (rc == PTAP_OK) rc = b->mem.get_n(&b->status, 1);
  if (rc == PTAP_OK && cudaMemsetAsync(b->status, 0, sizeof(int32_t), s) != cudaSuccess) rc = PTAP_ERR_CUDA;
  if (rc == PTAP_OK) rc = ptap::batch_create(b, plans, A, P, C_vals, s);
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
  if (b->n_fast + b->n_gen == 0) return PTAP_OK;
  return ptap::batch_launch(b, (cudaStream_t)stream);
}

extern "C" void ptap_batch_destroy(ptap_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->mem.stream);
  b->mem.release_all();
  delete b;
}
