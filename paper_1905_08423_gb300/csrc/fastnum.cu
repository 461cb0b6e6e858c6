// Host side of the class-program numeric kernel (owner mode, fast path).
// The device code is in fastkern.cuh; this file instantiates the interpreter
// kernel and launches either it or the plan's NVRTC-specialised kernel
// (jit.cu), whose classes run as straight-line code.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "fastkern.cuh"

namespace ptap {

using ptapk::FastArgs;
using ptapk::FCsr;

namespace {
struct NoSpecial {
  template <typename V>
  __device__ bool operator()(const FastArgs<V>&, int32_t, int32_t, int32_t, int32_t, int32_t, V*,
                             const int32_t*, int32_t, const int32_t*) const {
    return false;
  }
};
}  // namespace

// MaxT: the largest CTA the instantiation is compiled for (256, or 1024 for
// the large-chunk configurations, which cap registers at 64).
template <typename V, int MaxT>
__global__ void __launch_bounds__(MaxT) k_numeric_fast(FastArgs<V> a) {
  ptapk::fast_kernel_body<V>(a, NoSpecial());
}

template <typename V>
static FastArgs<V> fast_args(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C) {
  FastArgs<V> a;
  a.A = FCsr<V>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const V*)A->val};
  a.P = FCsr<V>{P->nrows, P->ncols, P->row_ptr, P->col_idx, (const V*)P->val};
  a.c_rp = p->c_rp;
  a.c_val = (V*)C;
  a.chunk_row = p->chunk_row;
  a.chunk_piece = p->chunk_piece;
  a.piece_f0 = p->piece_f0;
  a.piece_meta = p->piece_meta;
  a.frows = p->chunk_frows;
  a.pool = p->class_pool;
  a.class_off = p->class_off;
  a.nchunks = p->nchunks;
  a.CH = p->cfg.chunk_entries;
  a.max_rows = std::max(p->max_chunk_rows, 1);
  a.prog_cap = (p->class_maxlen + 15) & ~15;
  a.maxr = std::max(p->class_maxr, 1);
  a.work = p->work;
  a.chunk_order = p->chunk_order;
  a.rs_global = (V*)p->interp_rs;
  a.jit_slot = p->jit_slot;
  a.aq = p->aq;
  a.rec = p->rec;
  a.rec_off = p->rec_off;
  a.crows = p->compact ? p->chunk_crows : nullptr;
  a.row_loc = p->compact ? p->row_loc : nullptr;
  a.chunk_nnz = p->compact ? p->chunk_nnz : nullptr;
  a.loc_bits = p->loc_bits;
  return a;
}

template <typename V>
static size_t fast_smem(const ptap_plan* p, bool rs_in_smem = true) {
  return ptapk::fast_smem_bytes<V>(p->cfg.chunk_entries, p->cfg.block_threads, std::max(p->class_maxr, 1),
                                   std::max(p->max_chunk_rows, 1), (p->class_maxlen + 15) & ~15, rs_in_smem);
}

// The specialised kernel's carve-up: the interpreted classes keep their rows
// of A P in global scratch, and with piece records no row offsets are kept.
size_t jit_smem_for(const ptap_plan* p) {
  const int rows = p->rec ? 0 : std::max(p->max_chunk_rows, 1);
  const int maxr = std::max(p->class_maxr, 1), cap = (p->class_maxlen + 15) & ~15;
  return p->dtype == PTAP_F64
             ? ptapk::fast_smem_bytes<double>(p->cfg.chunk_entries, p->cfg.block_threads, maxr, rows, cap, false)
             : ptapk::fast_smem_bytes<float>(p->cfg.chunk_entries, p->cfg.block_threads, maxr, rows, cap, false);
}

// The dynamic schedule: chunks ordered by fine-row visits, longest first, and
// a zeroed counter pair.
static int prepare_schedule(ptap_plan* p) {
  if (p->work) return PTAP_OK;
  cudaStream_t s = p->stream;
  std::vector<int32_t> fptr(p->nchunks + 1);
  PTAP_CUDA(cudaMemcpyAsync(fptr.data(), p->chunk_fptr, fptr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> order(p->nchunks);
  for (int32_t c = 0; c < p->nchunks; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return fptr[x + 1] - fptr[x] > fptr[y + 1] - fptr[y];
  });
  PTAP_TRY(p->mem.get_n(&p->chunk_order, std::max<int64_t>(p->nchunks, 1)));
  PTAP_TRY(p->mem.get_n(&p->work, 2));
  PTAP_CUDA(cudaMemcpyAsync(p->chunk_order, order.data(), order.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  PTAP_CUDA(cudaMemsetAsync(p->work, 0, 2 * sizeof(int32_t), s));
  PTAP_CUDA(cudaStreamSynchronize(s));
  return PTAP_OK;
}

template <typename V>
static auto fast_kernel_for(const ptap_plan* p) {
  return p->cfg.block_threads > 256 ? k_numeric_fast<V, 1024> : k_numeric_fast<V, 256>;
}

// Occupancy of the interpreter kernel for a dynamic shared-memory size; 0 if
// it cannot launch.
template <typename V>
static int fast_occupancy(const ptap_plan* p, size_t smem) {
  int dev = 0, optin = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  PTAP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)optin) return 0;
  auto k = fast_kernel_for<V>(p);
  PTAP_TRY(grow_smem_limit((const void*)k, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, p->cfg.block_threads, smem));
  return per_sm;
}

// The interpreter keeps its rows of A P in shared memory when they fit beside
// the accumulator; otherwise (large CTAs and chunks) in a global scratch of
// 32 * maxr values per warp of each resident CTA.
template <typename V>
static int prepare_fast_t(ptap_plan* p) {
  size_t smem = fast_smem<V>(p, true);
  int per_sm = fast_occupancy<V>(p, smem);
  if (per_sm < 1) {
    smem = fast_smem<V>(p, false);
    per_sm = fast_occupancy<V>(p, smem);
    if (per_sm < 1) return PTAP_ERR_INVALID;
    const int64_t ctas = std::min<int64_t>(std::max(p->nchunks, 1), (int64_t)num_sms() * per_sm);
    PTAP_TRY(p->mem.get(&p->interp_rs, (size_t)ctas * p->cfg.block_threads * std::max(p->class_maxr, 1) *
                                           sizeof(V)));
  }
  p->num_smem = smem;
  p->num_per_sm = per_sm;
  return PTAP_OK;
}

// The cached index of the class-program kernels: aq[e] = P.rp[A.ci[e]].
__global__ void k_index_cache(const int32_t* __restrict__ Aci, const int32_t* __restrict__ Prp, int64_t nnz,
                              int32_t* __restrict__ aq) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    aq[e] = Prp[Aci[e]];
}

// Piece records (the indices cached per visit): the size of each piece's
// record in 16-byte units, na int32 and pI uint16 per lane.
__global__ void k_rec_sizes(const int32_t* __restrict__ meta, const uint8_t* __restrict__ pool,
                            const int32_t* __restrict__ class_off, int64_t npieces, int32_t* __restrict__ size16) {
  for (int64_t pc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pc < npieces;
       pc += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* g = pool + class_off[meta[pc] >> 6];
    size16[pc] = g[0] * 8 + g[2] * 4;
  }
}

// Fills the records, one warp per piece, the chunks strided over the grid:
// per lane the row starts of P for the entries of A(I,:), and the accumulator
// offset of each P(I,s)'s row in the piece's chunk (0xFFFF when the row lies
// outside it, or the lane is past the piece's rows).
__global__ void k_rec_fill(CsrI A, CsrI P, const int32_t* __restrict__ c_rp, const int32_t* __restrict__ chunk_row,
                           const int32_t* __restrict__ chunk_piece, const int32_t* __restrict__ piece_f0,
                           const int32_t* __restrict__ piece_meta, const int32_t* __restrict__ frows,
                           const uint8_t* __restrict__ pool, const int32_t* __restrict__ class_off,
                           const int32_t* __restrict__ rec_off, int32_t nchunks, int32_t* __restrict__ rec) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int32_t i0 = chunk_row[c], i1 = chunk_row[c + 1], base = c_rp[i0];
    for (int32_t pc = chunk_piece[c] + warp; pc < chunk_piece[c + 1]; pc += nw) {
      const int32_t meta = piece_meta[pc], f0 = piece_f0[pc];
      const bool valid = lane < (meta & 63);
      const int32_t I = frows[f0 + (valid ? lane : 0)];
      const uint8_t* g = pool + class_off[meta >> 6];
      const int na = g[0], pI = g[2];
      int32_t* q = rec + 4 * (int64_t)rec_off[pc];
      const int32_t ra = A.rp[I];
      for (int x = 0; x < na; ++x) q[x * 32 + lane] = P.rp[A.ci[ra + x]];
      uint16_t* o = (uint16_t*)(q + na * 32);
      const int32_t rp = P.rp[I];
      for (int t = 0; t < pI; ++t) {
        const int32_t i = P.ci[rp + t];
        o[t * 32 + lane] = valid && i >= i0 && i < i1 ? (uint16_t)(c_rp[i] - base) : (uint16_t)0xFFFF;
      }
    }
  }
}

// Piece records for a class-program plan with range chunks; *done says
// whether they were built (not when the chunks are compact, the offsets would
// not fit 16 bits, or the records would pass 32 GB).
static int build_records(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, cudaStream_t s, bool* done) {
  *done = false;
  if (p->compact || p->cfg.chunk_entries > 0xFFFF || p->npieces <= 0) return PTAP_OK;
  Scratch sc(&p->mem);
  int32_t* size16 = nullptr;
  PTAP_TRY(sc.get(&size16, p->npieces));
  const int grid = (int)std::min<int64_t>(ceil_div(p->npieces, 256), (int64_t)num_sms() * 8);
  k_rec_sizes<<<grid, 256, 0, s>>>(p->piece_meta, p->class_pool, p->class_off, p->npieces, size16);
  PTAP_LAUNCHED();
  PTAP_TRY(p->mem.get_n(&p->rec_off, p->npieces));
  int64_t total16 = 0;
  const int rc = exclusive_scan(p->mem, size16, p->rec_off, p->npieces, &total16, s);
  if (rc == PTAP_ERR_OVERFLOW) {
    p->mem.put(p->rec_off);
    p->rec_off = nullptr;
    return PTAP_OK;
  }
  PTAP_TRY(rc);
  PTAP_TRY(p->mem.get((void**)&p->rec, (size_t)std::max<int64_t>(total16, 1) * 16));
  k_rec_fill<<<num_sms() * 4, 256, 0, s>>>(CsrI{A->nrows, A->ncols, A->row_ptr, A->col_idx},
                                           CsrI{P->nrows, P->ncols, P->row_ptr, P->col_idx}, p->c_rp,
                                           p->chunk_row, p->chunk_piece, p->piece_f0, p->piece_meta,
                                           p->chunk_frows, p->class_pool, p->class_off, p->rec_off, p->nchunks,
                                           (int32_t*)p->rec);
  PTAP_LAUNCHED();
  p->rec_bytes = total16 * 16;
  *done = true;
  return PTAP_OK;
}

int build_index_cache(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, cudaStream_t s) {
  if (!p->fast || !p->cfg.cache_indices || p->aq || p->rec || p->nnz_a == 0) return PTAP_OK;
  if (p->cfg.cache_indices == 2) {
    bool done = false;
    PTAP_TRY(build_records(p, A, P, s, &done));
    if (done) return PTAP_OK;
  }
  PTAP_TRY(p->mem.get_n(&p->aq, p->nnz_a));
  k_index_cache<<<num_sms() * 8, 256, 0, s>>>(A->col_idx, P->row_ptr, p->nnz_a, p->aq);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

int jit_prepare(ptap_plan* p);  // jit.cu
int jit_launch(ptap_plan* p, void* fn, const void* args, int grid, cudaStream_t s);

int prepare_fast(ptap_plan* p) {
  PTAP_TRY(p->dtype == PTAP_F64 ? prepare_fast_t<double>(p) : prepare_fast_t<float>(p));
  PTAP_TRY(prepare_schedule(p));
  // optional: the interpreter runs if it fails; batch-only specialisation
  // leaves the compile to ptap_batch_create
  if (p->cfg.jit && p->cfg.jit_scope == 0) {
    PhaseRange r("ptap: specialise classes (NVRTC)", p->stream);
    jit_prepare(p);
  }
  return PTAP_OK;
}

template <typename V>
static int launch_fast_t(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  FastArgs<V> args = fast_args<V>(p, A, P, C);
  if (void* fn = p->jit_fn.load(std::memory_order_acquire)) {
    const int grid = (int)std::min<int64_t>(p->nchunks, (int64_t)num_sms() * p->jit_per_sm);
    if (grid <= 0) return PTAP_OK;
    args.rs_global = (V*)p->jit_rs;
    if (p->rec) args.max_rows = 0;  // the carve-up of jit_smem_for
    return jit_launch(p, fn, &args, grid, s);
  }
  const int grid = (int)std::min<int64_t>(p->nchunks, (int64_t)num_sms() * p->num_per_sm);
  if (grid <= 0) return PTAP_OK;
  fast_kernel_for<V>(p)<<<grid, p->cfg.block_threads, p->num_smem, s>>>(args);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

int numeric_fast(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  return p->dtype == PTAP_F64 ? launch_fast_t<double>(p, A, P, C, s) : launch_fast_t<float>(p, A, P, C, s);
}

}  // namespace ptap
