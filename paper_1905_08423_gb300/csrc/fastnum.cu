// Fast owner-mode numeric kernel: fine rows of one structure class in lockstep.
//
// Same product as the general owner kernel (Section 3, Eq. 9, Alg. 8): a CTA
// owns a chunk of coarse rows, accumulates C's values for it on chip and
// writes them once.  The difference is how a fine row's work is organised.
// The symbolic phase (classes.cu) grouped the fine rows visiting each chunk
// into runs of one structure class; here a warp takes 32 rows of a run, one
// per lane, and runs the class's program:
//
//   R(t) += A(I,k_a) P(k_a, b)    for each term (a, b), t = program slot  (Alg. 3)
//   C(i_s, sigma(s,t)) += P(I,i_s) R(t)   for i_s inside the chunk       (Alg. 8)
//
// Every index the lanes use is either loaded data (the value arrays and the
// row pointers) or the program, which is the same for all 32 lanes: the slot
// of each product in R and its position in C are offsets read from the
// program, so there is no hash table and no search, and C's column indices
// are never read.
#include <algorithm>

#include "owner.cuh"

namespace ptap {

template <typename V>
struct FastArgs {
  CsrV<V> A, P;
  const int32_t* c_rp;
  V* c_val;
  const int32_t* chunk_row;
  const int32_t* chunk_piece;
  const int32_t* piece_f0;
  const int32_t* piece_meta;
  const int32_t* frows;
  const uint8_t* pool;
  const int32_t* class_off;
  int32_t nchunks;
  int32_t CH;
  int32_t max_rows;
  int32_t prog_cap;  // bytes of program buffer per warp (multiple of 16)
  int32_t maxr;      // largest row of A P over the classes
};

// 32 fine rows [f, min(f+32, f1)) of one class, one per lane.  R is the
// lane's row of A P, held lane-major in shared memory (R[t*32 + lane]) so a
// product lands in its slot with no branch.
template <typename V>
__device__ __forceinline__ void fast_piece(const FastArgs<V>& a, const uint8_t* prog, V* R, int32_t f,
                                           int32_t f1, int32_t i0, int32_t i1, V* acc,
                                           const int32_t* roff) {
  const int lane = threadIdx.x & 31;
  const bool valid = f + lane < f1;
  // lanes past the run's end redo its first row and add nothing
  const int32_t I = a.frows[valid ? f + lane : f];
  const int na = prog[0], r = prog[1], pI = prog[2];
  const uint8_t* pa_sec = prog + 8;
  const uint64_t* t_sec = (const uint64_t*)(prog + 8 + ((na + 7) & ~7));
  const uint64_t* s_sec = t_sec + na;
  for (int t = 0; t < r; ++t) R[t * 32 + lane] = V(0);
  // row of A P (Alg. 3), four entries of A(I,:) at a time
  const int32_t ra = a.A.rp[I];
  for (int x0 = 0; x0 < na; x0 += 4) {
    int32_t k[4];
    V av[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (x0 + j < na) {
        k[j] = a.A.ci[ra + x0 + j];
        av[j] = a.A.val[ra + x0 + j];
      }
    int32_t pb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (x0 + j < na) pb[j] = a.P.rp[k[j]];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (x0 + j >= na) break;
      const int pa = pa_sec[x0 + j];
      const uint64_t tw = t_sec[x0 + j];
      V v[kFastMaxB];
#pragma unroll
      for (int b = 0; b < kFastMaxB; ++b)
        if (b < pa) v[b] = a.P.val[pb[j] + b];
#pragma unroll
      for (int b = 0; b < kFastMaxB; ++b) {
        if (b >= pa) break;
        const int t = (int)((tw >> (8 * b)) & 0xff);
        R[t * 32 + lane] += av[j] * v[b];
      }
    }
  }
  // outer product with P(I,:) into the chunk (Alg. 8)
  const int32_t rp = a.P.rp[I];
  int32_t cb[kFastMaxP];
  V ws[kFastMaxP];
#pragma unroll
  for (int s = 0; s < kFastMaxP; ++s) {
    cb[s] = -1;
    ws[s] = V(0);
    if (s < pI) {
      const int32_t i = a.P.ci[rp + s];
      ws[s] = a.P.val[rp + s];
      if (valid && i >= i0 && i < i1) cb[s] = roff[i - i0];
    }
  }
  for (int t = 0; t < r; ++t) {
    const V rt = R[t * 32 + lane];
    const uint64_t sw = s_sec[t];
#pragma unroll
    for (int s = 0; s < kFastMaxP; ++s) {
      if (s >= pI) break;
      if (cb[s] >= 0) atomicAdd(&acc[cb[s] + (int)((sw >> (8 * s)) & 0xff)], ws[s] * rt);
    }
  }
}

template <typename V>
__global__ void __launch_bounds__(256) k_numeric_fast(FastArgs<V> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int CHa = (a.CH + 3) & ~3;  // keeps the later regions 16-byte aligned
  V* acc = (V*)smraw;
  V* Rs = acc + CHa + (size_t)warp * 32 * a.maxr;
  int32_t* roff = (int32_t*)(acc + CHa + (size_t)nwarps * 32 * a.maxr);
  uint8_t* progs = (uint8_t*)(roff + ((a.max_rows + 1 + 3) & ~3));
  uint8_t* prog = progs + warp * a.prog_cap;
  for (int32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
    const int32_t i0 = a.chunk_row[c], i1 = a.chunk_row[c + 1];
    const int32_t base = a.c_rp[i0], nnz = a.c_rp[i1] - base;
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) acc[t] = V(0);
    for (int t = threadIdx.x; t <= i1 - i0; t += blockDim.x) roff[t] = a.c_rp[i0 + t] - base;
    __syncthreads();
    // the chunk's pieces (<= 32 rows of one class) go round-robin to the warps
    int32_t loaded = -1;
    const int32_t pe = a.chunk_piece[c + 1];
    for (int32_t pc = a.chunk_piece[c] + warp; pc < pe; pc += nwarps) {
      const int32_t meta = a.piece_meta[pc], f0 = a.piece_f0[pc];
      const int32_t cls = meta >> 6;
      if (cls != loaded) {
        __syncwarp();
        const uint8_t* src = a.pool + a.class_off[cls];
        for (int x = lane; x < a.prog_cap; x += 32) prog[x] = src[x];
        __syncwarp();
        loaded = cls;
      }
      fast_piece<V>(a, prog, Rs, f0, f0 + (meta & 63), i0, i1, acc, roff);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) a.c_val[base + t] = acc[t];
    __syncthreads();
  }
}

template <typename V>
static FastArgs<V> fast_args(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C) {
  FastArgs<V> a;
  a.A = CsrV<V>{A->nrows, A->ncols, A->row_ptr, A->col_idx, (const V*)A->val};
  a.P = CsrV<V>{P->nrows, P->ncols, P->row_ptr, P->col_idx, (const V*)P->val};
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
static size_t fast_smem(const ptap_plan* p, int threads) {
  const int prog_cap = (p->class_maxlen + 15) & ~15;
  const int rows = (std::max(p->max_chunk_rows, 1) + 1 + 3) & ~3;
  return ((size_t)((p->cfg.chunk_entries + 3) & ~3) + (size_t)threads * std::max(p->class_maxr, 1)) *
             sizeof(V) +
         (size_t)rows * 4 + (size_t)(threads / 32) * prog_cap;
}

template <typename V>
static int prepare_fast_t(ptap_plan* p) {
  const size_t smem = fast_smem<V>(p, p->cfg.block_threads);
  PTAP_CUDA(cudaFuncSetAttribute(k_numeric_fast<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_numeric_fast<V>,
                                                          p->cfg.block_threads, smem));
  if (per_sm < 1) return PTAP_ERR_INVALID;
  p->num_smem = smem;
  p->num_per_sm = per_sm;
  return PTAP_OK;
}

template <typename V>
static int launch_fast_t(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(p->nchunks, (int64_t)num_sms() * p->num_per_sm);
  if (grid <= 0) return PTAP_OK;
  k_numeric_fast<V><<<grid, p->cfg.block_threads, p->num_smem, s>>>(fast_args<V>(p, A, P, C));
  PTAP_LAUNCHED();
  return PTAP_OK;
}

int prepare_fast(ptap_plan* p) {
  return p->dtype == PTAP_F64 ? prepare_fast_t<double>(p) : prepare_fast_t<float>(p);
}

int numeric_fast(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s) {
  return p->dtype == PTAP_F64 ? launch_fast_t<double>(p, A, P, C, s) : launch_fast_t<float>(p, A, P, C, s);
}

}  // namespace ptap
