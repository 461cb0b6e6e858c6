// Device code of the class-program numeric kernel (owner mode, fast path).
//
// This header is compiled twice: by nvcc into libptap (the interpreter kernel
// k_numeric_fast) and, at symbolic time, by NVRTC together with generated
// straight-line code for the plan's most frequent classes (jit.cu).  It
// therefore includes no system header under NVRTC and holds device code only.
//
// The product (Section 3, Eq. 9, Alg. 8): a CTA owns a chunk of coarse rows,
// accumulates C's values for it on chip and writes them once.  The fine rows
// visiting the chunk come in pieces of at most 32 rows of one structure
// class; a warp runs one piece, one row per lane:
//
//   R(t) += A(I,k_a) P(k_a, b)            for each product (a, b)       (Alg. 3)
//   C(i_s, sigma(s,t)) += P(I,i_s) R(t)    for i_s inside the chunk     (Alg. 8)
//
// Program layout (bytes, see classes.cu): [0] na, [1] r, [2] pI, [8..8+A8)
// p_a, then t(a,b) at a*8+b, then sigma at t*8+s.
#pragma once

#ifdef __CUDACC_RTC__
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef decltype(sizeof(0)) size_t;
#else
#include <stdint.h>
#endif

namespace ptapk {

constexpr int kMaxB = 8;  // entries of each P(k,:) a class may reach
constexpr int kMaxP = 8;  // entries of P(I,:)

template <typename V>
struct FCsr {
  int32_t nrows, ncols;
  const int32_t* rp;
  const int32_t* ci;
  const V* val;
};

template <typename V>
struct FastArgs {
  FCsr<V> A, P;
  const int32_t* c_rp;
  V* c_val;
  const int32_t* chunk_row;
  const int32_t* chunk_piece;
  const int32_t* piece_f0;
  const int32_t* piece_meta;  // class << 6 | rows
  const int32_t* frows;
  const uint8_t* pool;
  const int32_t* class_off;
  int32_t nchunks;
  int32_t CH;
  int32_t max_rows;
  int32_t prog_cap;  // bytes of program buffer per warp (multiple of 16)
  int32_t maxr;      // largest row of A P over the classes
  // Optional dynamic schedule: when `work` is set, CTAs take chunks in the
  // order `chunk_order` (longest first) from the counter work[0]; the last CTA
  // to finish resets work[0] and work[1] to zero for the next launch.
  int32_t* work;
  const int32_t* chunk_order;
  // Optional global scratch for the interpreter's rows of A P (32 * maxr
  // values per warp of each resident CTA); null keeps them in shared memory.
  V* rs_global;
  // Plan-time specialised code: the compiled-code number of each class, or
  // -1 (null without compiled code).
  const int32_t* jit_slot;
  // Optional cached index: aq[e] = P.rp[A.ci[e]] for every entry e of A
  // (null: looked up through A.ci).
  const int32_t* aq;
  // Optional piece records (cached per visit instead of per entry of A):
  // piece pc's record starts at rec + 4 * rec_off[pc] and holds, lane-major,
  //   q[x * 32 + lane] = P.rp[A.ci[A.rp[I] + x]]   for x < na       (int32)
  //   o[s * 32 + lane] = accumulator offset of the row P.ci[P.rp[I] + s] in
  //                      the piece's chunk, 0xFFFF outside it or past the
  //                      piece's rows                   for s < pI       (uint16)
  // for the lane's fine row I, so a warp reads them with coalesced loads.
  // Null: aq, or A.ci and P's row starts.  Range chunks only.
  const int32_t* rec;
  const int32_t* rec_off;
  // Optional compact chunks.  When row_loc is set, the coarse rows of chunk c
  // are crows[chunk_row[c] .. chunk_row[c+1]) (ascending), row_loc[i] =
  // chunk << loc_bits | offset of row i's first entry in that chunk's
  // accumulator, and chunk_nnz[c] is the chunk's entries.  Null: chunk c is
  // the range of coarse rows [chunk_row[c], chunk_row[c+1]).
  const int32_t* crows;
  const int32_t* row_loc;
  const int32_t* chunk_nnz;
  int32_t loc_bits;
};

// Adds v to *p, p in shared memory.  A relaxed reduction: the barrier that
// ends the chunk orders it before the accumulator is read.
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.shared.add.f64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "d"(v) : "memory");
}

// *p += w * r for p in shared memory (one outer-product term of Alg. 8).
// Each form is the one measured fastest where it is used:
//  - compiled classes: a shared-memory reduction (red.shared.add), FP32 and FP64;
//  - interpreter, FP32: atomicAdd (fewer registers in its loops);
//  - interpreter, FP64: a compare-and-swap loop whose new value is
//    fma(w, r, old) -- one FP64 operation a term on a part whose FP64 pipe
//    bounds this path (and one rounding).  Lock-free: a failed swap means
//    another thread's update went in.
__device__ __forceinline__ void acc_fma(float* p, float w, float r) { red_add(p, w * r); }
__device__ __forceinline__ void acc_fma(double* p, double w, double r) { red_add(p, w * r); }
__device__ __forceinline__ void interp_add(float* p, float w, float r) { atomicAdd(p, w * r); }
__device__ __forceinline__ void interp_add(double* p, double w, double r) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned long long old;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(old) : "r"(a) : "memory");
  for (;;) {
    const unsigned long long nv =
        (unsigned long long)__double_as_longlong(fma(w, r, __longlong_as_double((long long)old)));
    unsigned long long got;
    asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(got) : "r"(a), "l"(old), "l"(nv) : "memory");
    if (got == old) break;
    old = got;
  }
}

// Interpreter: 32 fine rows [f, min(f+32, f1)) of one class, one per lane.
// R is the lane's row of A P, lane-major in shared memory (R[t*32 + lane]).
// The chunk is the coarse rows [i0, i1) with row offsets roff, or, with
// compact chunks, chunk number i0 (i1 and roff unused).
template <typename V>
__device__ __forceinline__ void fast_piece(const FastArgs<V>& a, const uint8_t* prog, V* R, int32_t f,
                                           int32_t f1, int32_t i0, int32_t i1, V* acc,
                                           const int32_t* roff, int32_t I, const int32_t* rec) {
  const int lane = threadIdx.x & 31;
  const bool valid = f + lane < f1;
  // lanes past the piece's end redo its first row (I) and add nothing
  const int na = prog[0], r = prog[1], pI = prog[2];
  const uint8_t* pa_sec = prog + 8;
  const uint64_t* t_sec = (const uint64_t*)(prog + 8 + ((na + 7) & ~7));
  const uint64_t* s_sec = t_sec + na;
  for (int t = 0; t < r; ++t) R[t * 32 + lane] = V(0);
  // row of A P (Alg. 3), four entries of A(I,:) at a time
  const int32_t ra = a.A.rp[I];
  for (int x0 = 0; x0 < na; x0 += 4) {
    int32_t k[4] = {0, 0, 0, 0};
    V av[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (x0 + j < na) {
        if (!a.aq && !rec) k[j] = a.A.ci[ra + x0 + j];
        av[j] = a.A.val[ra + x0 + j];
      }
    int32_t pb[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (x0 + j < na)
        pb[j] = rec ? rec[(x0 + j) * 32 + lane] : a.aq ? a.aq[ra + x0 + j] : a.P.rp[k[j]];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (x0 + j >= na) break;
      const int pa = pa_sec[x0 + j];
      const uint64_t tw = t_sec[x0 + j];
      V v[kMaxB];
#pragma unroll
      for (int b = 0; b < kMaxB; ++b)
        if (b < pa) v[b] = a.P.val[pb[j] + b];
#pragma unroll
      for (int b = 0; b < kMaxB; ++b) {
        if (b >= pa) break;
        const int t = (int)((tw >> (8 * b)) & 0xff);
        R[t * 32 + lane] += av[j] * v[b];
      }
    }
  }
  // outer product with P(I,:) into the chunk (Alg. 8)
  const int32_t rp = a.P.rp[I];
  int32_t cb[kMaxP];
  V ws[kMaxP];
#pragma unroll
  for (int s = 0; s < kMaxP; ++s) {
    cb[s] = -1;
    ws[s] = V(0);
    if (s < pI) {
      ws[s] = a.P.val[rp + s];
      if (rec) {
        const int32_t o = ((const uint16_t*)(rec + na * 32))[s * 32 + lane];
        if (o != 0xFFFF) cb[s] = o;
      } else if (valid) {
        const int32_t i = a.P.ci[rp + s];
        if (a.row_loc) {
          const int32_t l = a.row_loc[i];
          if ((l >> a.loc_bits) == i0) cb[s] = l & ((1 << a.loc_bits) - 1);
        } else if (i >= i0 && i < i1) {
          cb[s] = roff[i - i0];
        }
      }
    }
  }
  for (int t = 0; t < r; ++t) {
    const V rt = R[t * 32 + lane];
    const uint64_t sw = s_sec[t];
#pragma unroll
    for (int s = 0; s < kMaxP; ++s) {
      if (s >= pI) break;
      if (cb[s] >= 0) interp_add(&acc[cb[s] + (int)((sw >> (8 * s)) & 0xff)], ws[s], rt);
    }
  }
}

// Shared-memory carve-up: accumulator | interpreter R rows (unless they live
// in global scratch) | row offsets | per-warp program buffers; every region
// 16-byte aligned.  max_rows = 0 with piece records, which carry the
// accumulator offsets themselves.  What is not carved stays L1.
template <typename V>
__host__ __device__ inline size_t fast_smem_bytes(int CH, int threads, int maxr, int max_rows,
                                                  int prog_cap, bool rs_in_smem = true) {
  const int CHa = (CH + 3) & ~3;
  const int rows = (max_rows + 1 + 3) & ~3;
  return ((size_t)CHa + (rs_in_smem ? (size_t)threads * maxr : 0)) * sizeof(V) + (size_t)rows * 4 +
         (size_t)(threads / 32) * prog_cap;
}

// Per-warp pointers into the shared-memory carve-up (dims are the largest
// over the problems a kernel serves: one product, or a batch).
template <typename V>
struct FastSmem {
  V* acc;
  V* Rs;
  int32_t* roff;
  uint8_t* prog;
  __device__ FastSmem(unsigned char* raw, int CH, int maxr, int max_rows, int prog_cap,
                      V* rs_global = nullptr) {
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int CHa = (CH + 3) & ~3;
    acc = (V*)raw;
    if (rs_global) {
      Rs = rs_global + ((size_t)blockIdx.x * nwarps + warp) * 32 * maxr;
      roff = (int32_t*)(acc + CHa);
    } else {
      Rs = acc + CHa + (size_t)warp * 32 * maxr;
      roff = (int32_t*)(acc + CHa + (size_t)nwarps * 32 * maxr);
    }
    prog = (uint8_t*)(roff + ((max_rows + 1 + 3) & ~3)) + warp * prog_cap;
  }
};

// One chunk c of a product.  `special(a, slot, f, f1, i0, i1, acc, roff, I, rec)`
// runs a piece whose class has compiled code number `slot` (jit_slot of its
// class, -1 for none) and returns true; otherwise the interpreter runs it from
// the class's program.  slot, the lane's fine row I and the piece's record
// rec (or null) are loaded one piece ahead.  With compact chunks
// i0 is the chunk number and the values go back to C row by row.
template <typename V, typename Special>
__device__ __forceinline__ void fast_chunk(const FastArgs<V>& a, int32_t c, FastSmem<V>& sm,
                                           Special special) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  V* acc = sm.acc;
  int32_t* roff = sm.roff;
  const bool compact = a.row_loc != nullptr;
  int32_t i0, i1, base = 0, nnz;
  if (compact) {
    i0 = c;
    i1 = 0;
    nnz = a.chunk_nnz[c];
  } else {
    i0 = a.chunk_row[c];
    i1 = a.chunk_row[c + 1];
    base = a.c_rp[i0];
    nnz = a.c_rp[i1] - base;
  }
  for (int t = threadIdx.x; t < nnz; t += blockDim.x) acc[t] = V(0);
  if (!compact && !a.rec)
    for (int t = threadIdx.x; t <= i1 - i0; t += blockDim.x) roff[t] = a.c_rp[i0 + t] - base;
  __syncthreads();
  // the chunk's pieces (<= 32 rows of one class) go round-robin to the warps
  int32_t loaded = -1;
  const int32_t pe = a.chunk_piece[c + 1];
  int32_t pc = a.chunk_piece[c] + warp;
  // software pipeline over this warp's pieces: the descriptor two pieces
  // ahead and the fine row one piece ahead are loaded while a piece runs
  int32_t meta = 0, f0 = 0, metan = 0, f0n = 0, I = 0, ro = 0;
  if (pc < pe) {
    meta = a.piece_meta[pc];
    f0 = a.piece_f0[pc];
  }
  if (pc + nwarps < pe) {
    metan = a.piece_meta[pc + nwarps];
    f0n = a.piece_f0[pc + nwarps];
  }
  int32_t sl = -1;
  if (pc < pe) {
    I = a.frows[f0 + lane < f0 + (meta & 63) ? f0 + lane : f0];
    if (a.rec) ro = a.rec_off[pc];
    if (a.jit_slot) sl = a.jit_slot[meta >> 6];
  }
  for (; pc < pe; pc += nwarps) {
    int32_t In = 0, metann = 0, f0nn = 0, ron = 0, sln = -1;
    if (pc + nwarps < pe) {
      In = a.frows[f0n + lane < f0n + (metan & 63) ? f0n + lane : f0n];
      if (a.rec) ron = a.rec_off[pc + nwarps];
      if (a.jit_slot) sln = a.jit_slot[metan >> 6];
    }
    if (pc + 2 * nwarps < pe) {
      metann = a.piece_meta[pc + 2 * nwarps];
      f0nn = a.piece_f0[pc + 2 * nwarps];
    }
    const int32_t cls = meta >> 6, f1 = f0 + (meta & 63);
    const int32_t* rec = a.rec ? a.rec + 4 * (size_t)ro : nullptr;
    if (!special(a, sl, f0, f1, i0, i1, acc, roff, I, rec)) {
      if (cls != loaded) {
        // programs start on 8-byte boundaries and the pool is padded past the
        // longest, so the copy moves prog_cap bytes as 8-byte words
        __syncwarp();
        const uint2* src = (const uint2*)(a.pool + a.class_off[cls]);
        for (int x = lane; x < a.prog_cap / 8; x += 32) ((uint2*)sm.prog)[x] = src[x];
        __syncwarp();
        loaded = cls;
      }
      fast_piece<V>(a, sm.prog, sm.Rs, f0, f1, i0, i1, acc, roff, I, rec);
    }
    meta = metan;
    f0 = f0n;
    metan = metann;
    f0n = f0nn;
    I = In;
    ro = ron;
    sl = sln;
  }
  __syncthreads();
  if (compact) {
    // 32 coarse rows per warp step: each lane looks up one row's place in C
    // and in the accumulator, then the warp copies the rows one by one
    const int32_t mask = (1 << a.loc_bits) - 1;
    const int32_t r1 = a.chunk_row[c + 1];
    for (int32_t j0 = a.chunk_row[c] + warp * 32; j0 < r1; j0 += nwarps * 32) {
      int32_t b = 0, len = 0, off = 0;
      if (j0 + lane < r1) {
        const int32_t i = a.crows[j0 + lane];
        b = a.c_rp[i];
        len = a.c_rp[i + 1] - b;
        off = a.row_loc[i] & mask;
      }
      const int nr = min(32, r1 - j0);
      for (int r = 0; r < nr; ++r) {
        const int32_t br = __shfl_sync(0xffffffffu, b, r), lr = __shfl_sync(0xffffffffu, len, r),
                      orr = __shfl_sync(0xffffffffu, off, r);
        for (int32_t x = lane; x < lr; x += 32) a.c_val[br + x] = acc[orr + x];
      }
    }
  } else {
    for (int t = threadIdx.x; t < nnz; t += blockDim.x) a.c_val[base + t] = acc[t];
  }
  __syncthreads();
}

// The single-product kernel body: chunks from a counter, longest first (or,
// without the plan's counter, strided over the grid).
template <typename V, typename Special>
__device__ __forceinline__ void fast_kernel_body(const FastArgs<V>& a, Special special) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t next;
  FastSmem<V> sm(smraw, a.CH, a.maxr, a.max_rows, a.prog_cap, a.rs_global);
  if (!a.work) {
    for (int32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) fast_chunk<V>(a, c, sm, special);
    return;
  }
  // chunks from a shared counter, longest first: no CTA idles while others
  // still hold several chunks
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(&a.work[0], 1);
    __syncthreads();
    const int32_t t = next;
    __syncthreads();
    if (t >= a.nchunks) break;
    fast_chunk<V>(a, a.chunk_order ? a.chunk_order[t] : t, sm, special);
  }
  // the last CTA to leave puts the counters back to zero for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.work[1], 1) == (int32_t)gridDim.x - 1) {
      atomicExch(&a.work[0], 0);
      atomicExch(&a.work[1], 0);
    }
  }
}

// The batched kernel body: chunks of many products from one queue of
// (problem, chunk) items, longest first, popped with the counter *counter
// (zero before the launch).  Each problem has its own descriptor; the CTA
// carve-up is sized for the largest chunk, row of A P, chunk row count and
// program over the problems, and the interpreter's rows of A P go to `rs`
// (global scratch) when it is not null.  No CTA waits on another.
template <typename V, typename Special>
__device__ __forceinline__ void fast_batch_body(const FastArgs<V>* __restrict__ probs,
                                                const int32_t* __restrict__ items, int32_t nitems,
                                                int32_t* counter, int CH, int maxr, int max_rows,
                                                int prog_cap, V* rs, Special special) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t item;
  FastSmem<V> sm(smraw, CH, maxr, max_rows, prog_cap, rs);
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    const int32_t it = item;
    __syncthreads();
    if (it >= nitems) break;
    const FastArgs<V> a = probs[items[2 * it]];
    fast_chunk<V>(a, items[2 * it + 1], sm, special);
  }
}

}  // namespace ptapk
