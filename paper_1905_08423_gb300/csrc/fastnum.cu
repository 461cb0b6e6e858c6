// Host side of the class-program numeric kernel (owner mode, fast path).
// The device code is in fastkern.cuh; this file instantiates the interpreter
// kernel and launches either it or the plan's NVRTC-specialised kernel
// (jit.cu), whose classes run as straight-line code.
#include <algorithm>

#include "common.cuh"
#include "fastkern.cuh"

namespace ptap {

using ptapk::FastArgs;
using ptapk::FCsr;

namespace {
struct NoSpecial {
  template <typename V>
  __device__ bool operator()(const FastArgs<V>&, int32_t, int32_t, int32_t, int32_t, int32_t, V*,
                             const int32_t*) const {
    return false;
  }
};
}  // namespace

template <typename V>
__global__ void __launch_bounds__(256) k_numeric_fast(FastArgs<V> a) {
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
  return a;
}

template <typename V>
static size_t fast_smem(const ptap_plan* p) {
  return ptapk::fast_smem_bytes<V>(p->cfg.chunk_entries, p->cfg.block_threads, std::max(p->class_maxr, 1),
                                   std::max(p->max_chunk_rows, 1), (p->class_maxlen + 15) & ~15);
}

size_t fast_smem_for(const ptap_plan* p) {
  return p->dtype == PTAP_F64 ? fast_smem<double>(p) : fast_smem<float>(p);
}

template <typename V>
static int prepare_fast_t(ptap_plan* p) {
  const size_t smem = fast_smem<V>(p);
  PTAP_CUDA(cudaFuncSetAttribute(k_numeric_fast<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_numeric_fast<V>, p->cfg.block_threads,
                                                          smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  p->num_smem = smem;
  p->num_per_sm = per_sm;
  return PTAP_OK;
}

int jit_prepare(ptap_plan* p);  // jit.cu
int jit_launch(ptap_plan* p, const void* args, int grid, cudaStream_t s);

int prepare_fast(ptap_plan* p) {
  PTAP_TRY(p->dtype == PTAP_F64 ? prepare_fast_t<double>(p) : prepare_fast_t<float>(p));
  if (p->cfg.jit) jit_prepare(p);  // optional: the interpreter runs if it fails
  return PTAP_OK;
}

template <typename V>
static int launch_fast_t(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  const FastArgs<V> args = fast_args<V>(p, A, P, C);
  if (p->jit_fn) {
    const int grid = (int)std::min<int64_t>(p->nchunks, (int64_t)num_sms() * p->jit_per_sm);
    if (grid <= 0) return PTAP_OK;
    return jit_launch(p, &args, grid, s);
  }
  const int grid = (int)std::min<int64_t>(p->nchunks, (int64_t)num_sms() * p->num_per_sm);
  if (grid <= 0) return PTAP_OK;
  k_numeric_fast<V><<<grid, p->cfg.block_threads, p->num_smem, s>>>(args);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

int numeric_fast(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  return p->dtype == PTAP_F64 ? launch_fast_t<double>(p, A, P, C, s) : launch_fast_t<float>(p, A, P, C, s);
}

}  // namespace ptap
