// Internal declarations shared by the translation units of libptap.
// Not part of the public ABI (that is include/ptap.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cstdio>
#include <thread>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "ptap.h"

namespace ptap {

// Named range for profilers (NVTX): a timeline shows the library's phases.
// It costs nothing unless a profiling tool is attached.
// With PTAP_PROFILE set, the host time of every range (phases end with a
// stream synchronisation where their results are needed) goes to stderr.
bool profile_enabled();
void profile_report(const char* name, double ms);
struct Range {
  explicit Range(const char* n) : name(n) {
    nvtxRangePushA(n);
    if (profile_enabled()) t0 = std::chrono::steady_clock::now();
  }
  ~Range() {
    nvtxRangePop();
    if (profile_enabled())
      profile_report(name, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  }
  const char* name;
  std::chrono::steady_clock::time_point t0{};
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// A range whose profiled time includes the work it queued on stream `s`.
struct PhaseRange : Range {
  PhaseRange(const char* n, cudaStream_t st) : Range(n), s(st) {}
  ~PhaseRange() {
    if (profile_enabled()) cudaStreamSynchronize(s);
  }
  cudaStream_t s;
};

// ---------------------------------------------------------------------------
// error handling: no exception crosses the ABI; internal code returns codes.
// ---------------------------------------------------------------------------
#define PTAP_TRY(expr)            \
  do {                            \
    int _rc = (expr);             \
    if (_rc != PTAP_OK) return _rc; \
  } while (0)

#define PTAP_CUDA(expr)                                   \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) {                              \
      ptap::note_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return PTAP_ERR_CUDA;                               \
    }                                                     \
  } while (0)

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Raises the dynamic shared-memory limit of kernel `fn` on the current device
// to at least `bytes`, never lowering it: plans built earlier may launch the
// same kernel with a larger carve-up than the plan being built now.
int grow_smem_limit(const void* fn, int bytes);

// Launch check: a bad launch configuration is a CUDA error of this call.
#define PTAP_LAUNCHED() PTAP_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// device memory: every library allocation goes through one tracker so that a
// plan can report its live and peak bytes (the memory the paper compares).
// ---------------------------------------------------------------------------
struct Tracker {
  ptap_allocator user{};
  bool has_user = false;
  cudaStream_t stream = nullptr;
  int64_t live = 0, peak = 0;
  std::unordered_map<void*, size_t> sizes;

  void init(const ptap_allocator* a, cudaStream_t s) {
    stream = s;
    if (a && a->alloc && a->free) {
      user = *a;
      has_user = true;
    }
  }
  // Returns PTAP_OK and *p, or PTAP_ERR_OOM.  Zero-byte requests give a
  // small real allocation so that pointers are never NULL.
  int get(void** p, size_t bytes) {
    size_t b = bytes ? bytes : 16;
    b = (b + 255) & ~size_t(255);
    void* q = nullptr;
    if (has_user) {
      q = user.alloc(b, (void*)stream, user.ctx);
    } else if (cudaMallocAsync(&q, b, stream) != cudaSuccess) {
      cudaGetLastError();
      q = nullptr;
    }
    if (!q) return PTAP_ERR_OOM;
    sizes[q] = b;
    live += (int64_t)b;
    if (live > peak) peak = live;
    *p = q;
    return PTAP_OK;
  }
  template <typename T>
  int get_n(T** p, int64_t n) {
    return get((void**)p, (size_t)(n < 0 ? 0 : n) * sizeof(T));
  }
  void put(void* p) {
    if (!p) return;
    auto it = sizes.find(p);
    size_t b = it == sizes.end() ? 0 : it->second;
    if (it != sizes.end()) sizes.erase(it);
    live -= (int64_t)b;
    if (has_user) user.free(p, b, (void*)stream, user.ctx);
    else cudaFreeAsync(p, stream);
  }
  void release_all() {
    for (auto& kv : sizes) {
      if (has_user) user.free(kv.first, kv.second, (void*)stream, user.ctx);
      else cudaFreeAsync(kv.first, stream);
    }
    sizes.clear();
    live = 0;
  }
};

// RAII scratch for the duration of one call.
struct Scratch {
  Tracker* t;
  std::vector<void*> bufs;
  explicit Scratch(Tracker* tr) : t(tr) {}
  template <typename T>
  int get(T** p, int64_t n) {
    int rc = t->get_n(p, n);
    if (rc == PTAP_OK) bufs.push_back((void*)*p);
    return rc;
  }
  void release(void* p) {
    for (auto& b : bufs)
      if (b == p) {
        t->put(p);
        b = nullptr;
      }
  }
  ~Scratch() {
    for (void* b : bufs)
      if (b) t->put(b);
  }
};

// ---------------------------------------------------------------------------
// resolved configuration
// ---------------------------------------------------------------------------
struct Config {
  int mode = PTAP_MODE_OWNER;
  int chunk_entries = 0;      // 0: chosen at symbolic time
  int class_programs = 1;     // fast path by fine-row classes where the patterns allow
  int visit_block_log2 = 0;   // fast path visit order: blocks of 2^b fine rows (0 = class-major)
  int jit = 0;                // specialise the most frequent classes with NVRTC
  int jit_max_classes = 8;
  int jit_scope = 0;          // 0: the plan's own kernel; 1: only batches compile code
  int jit_async = 0;          // compile the plan's kernel in a background thread
  int block_threads = 256;
  int group_lanes = 8;
  int ap_slots = 64;
  int debug_checks = 0;
  int force_spill = 0;
  int cache_indices = 0;      // store P's row start for every entry of A (fast path)
  int general_kernel = 0;     // general path: 0 sort-based (warp per row), 1 hash groups
  int compact_chunks = 0;     // > 0: chunks grown over C's graph, by runs of this many rows
};

Config resolve_config(const ptap_config* c);

// ---------------------------------------------------------------------------
// device-side CSR views
// ---------------------------------------------------------------------------
struct CsrI {  // pattern only
  int32_t nrows, ncols;
  const int32_t* rp;
  const int32_t* ci;
};
template <typename V>
struct CsrV {
  int32_t nrows, ncols;
  const int32_t* rp;
  const int32_t* ci;
  const V* val;
};

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct TwoStepData;
struct HostStage;

}  // namespace ptap

struct ptap_plan {
  int kind = 0;  // 0 all-at-once, 1 two-step
  int dtype = PTAP_F64;
  int32_t n = 0, m = 0;
  int64_t nnz_a = 0, nnz_p = 0, nnz_c = 0;
  ptap::Tracker mem;
  cudaStream_t stream = nullptr;
  ptap::Config cfg;
  int64_t symbolic_peak = 0;
  int32_t spill_rows = 0;

  int32_t* c_rp = nullptr;  // C pattern (plan-owned)
  int32_t* c_ci = nullptr;

  // owner-mode numeric schedule
  int32_t nchunks = 0, nheavy = 0, max_chunk_rows = 0, max_chunk_nnz = 0;
  int32_t* chunk_row = nullptr;   // [nchunks+1] first coarse row of each chunk (ranges), or
                                  // first entry of the chunk in chunk_crows (compact chunks)
  // compact chunks (symbolic.cu): rows of each chunk, ascending; per coarse
  // row its chunk and accumulator offset packed as chunk << loc_bits | offset;
  // C entries per chunk
  bool compact = false;
  int32_t loc_bits = 0;
  int32_t* chunk_crows = nullptr;
  int32_t* row_loc = nullptr;
  int32_t* chunk_nnz = nullptr;
  int32_t* chunk_fptr = nullptr;  // [nchunks+1] offsets into chunk_frows
  int32_t* chunk_frows = nullptr; // fine rows visited per chunk, ascending
  int64_t nfrows = 0;

  int32_t* status = nullptr;  // device status word (PTAP_* code, 0 = ok)

  // launch configuration of the numeric kernel, settled at symbolic time
  size_t num_smem = 0;
  int num_per_sm = 0;
  // dynamic chunk schedule of the class-program kernels: a counter pair
  // (zero between launches) and the chunks longest first
  int32_t* work = nullptr;
  int32_t* chunk_order = nullptr;

  // fine-row classes for the fast numeric path (classes.cu)
  int fast = 0;
  int32_t nclasses = 0, nseg = 0, class_maxr = 0, class_maxlen = 0, class_maxa = 0;
  int64_t npieces = 0;
  int32_t* piece_f0 = nullptr;    // [npieces] first visit (index into chunk_frows) of each piece
  int32_t* piece_meta = nullptr;  // [npieces] class << 6 | rows (1..32)
  int32_t* chunk_piece = nullptr; // [nchunks+1] first piece of each chunk

  // plan-time specialised kernel (jit.cu); null when the interpreter runs
  // set (release) once the specialised code is loaded: at symbolic time, or
  // by jit_thread when the compile runs in the background (specialize_async);
  // launches read it (acquire) and run the interpreter until then
  std::atomic<void*> jit_fn{nullptr};
  std::thread* jit_thread = nullptr;
  void* jit_rs = nullptr;  // global scratch for the interpreted classes' rows of A P
  int32_t* jit_slot = nullptr;  // [nclasses] compiled-code number of each class, or -1
  int32_t* aq = nullptr;        // [nnz(A)] P.rp[A.ci[e]] when indices are cached
  // piece records (indices cached per visit, lane-major; fastkern.cuh has
  // the layout): record pc starts at rec + 4 * rec_off[pc]
  int32_t* rec = nullptr;
  int32_t* rec_off = nullptr;
  int64_t rec_bytes = 0;
  // 0: no cached indices, 1: aq, 2: piece records
  int index_mode() const { return rec ? 2 : aq ? 1 : 0; }
  void* interp_rs = nullptr;  // the same for the interpreter kernel, when shared memory is short
  size_t jit_smem = 0;
  int jit_per_sm = 0, jit_classes = 0;
  double jit_coverage = 0.0, jit_ms = 0.0;
  uint8_t* class_pool = nullptr; // class programs (signatures), see classes.cu
  int32_t* class_off = nullptr;  // [nclasses] offset of each program in the pool

  ptap::TwoStepData* two = nullptr;
  ptap::HostStage* host = nullptr;  // staging of ptap_numeric_host (host.cu)
};

struct ptap_batch {
  ptap::Tracker mem;
  int dtype = PTAP_F64;
  int32_t count = 0;
  int32_t* status = nullptr;
  int32_t* d_counter = nullptr;  // two counters: class-program items, general items
  // Problems whose plans run class programs go through the class-program
  // batch kernel (interpreted, or specialised for the batch with NVRTC); the
  // others through the general owner-mode batch kernel.  Each kind has its
  // own queue of (problem, chunk) items, longest first.
  int64_t n_fast = 0, n_gen = 0;
  void* d_desc_fast = nullptr;  // FastArgs per problem (class-program problems)
  void* d_desc_gen = nullptr;   // NumArgs per problem (general problems)
  int32_t* d_items_fast = nullptr;
  int32_t* d_items_gen = nullptr;
  // class-program kernel
  int fast_threads = 256, fast_ch = 0, fast_maxr = 1, fast_prog_cap = 16, fast_max_rows = 1;
  size_t fast_smem = 0;
  int fast_grid = 0;
  void* fast_rs = nullptr;   // global scratch for interpreted rows of A P (specialised kernel)
  void* jit_fn = nullptr;    // ptap_jit_batch, or null: the interpreter kernel runs
  int jit_classes = 0;
  double jit_coverage = 0.0;
  // general kernel
  ptap::Config cfg;          // lanes per fine row, hash slots, chunk size (largest), 256 threads
  int32_t max_chunk_rows = 1;
  size_t gen_smem = 0;
  int gen_grid = 0;
};

namespace ptap {

// ---------------------------------------------------------------------------
// shared host helpers (implemented in the .cu files named)
// ---------------------------------------------------------------------------
// scan.cu: exclusive scan of n int32 counts into out[0..n] (out[n] = total);
// PTAP_ERR_OVERFLOW if the total reaches 2^31.  *total receives the total
// (synchronises the stream when total != nullptr).
int exclusive_scan(Tracker& mem, const int32_t* in, int32_t* out, int64_t n,
                   int64_t* total, cudaStream_t s);
// scan.cu: sorts each segment [ptr[r], ptr[r+1]) of keys ascending (and the
// optional companion values alongside).
int segmented_sort(Tracker& mem, const int32_t* ptr, int32_t nseg, int32_t* keys,
                   int32_t* vals, int32_t max_len, cudaStream_t s);
// symbolic.cu: transpose of a CSR pattern: tp (ncols+1), tj (nnz) fine-row
// ids per column sorted ascending, and tperm (nnz, optional) = position in
// the source of each transposed entry.
int transpose_pattern(Tracker& mem, const CsrI& M, int32_t* tp, int32_t* tj,
                      int32_t* tperm, cudaStream_t s);
// validation of a CSR input (device); returns PTAP_ERR_INVALID on a bad matrix.
int validate_csr(Tracker& mem, const ptap_csr* M, cudaStream_t s);
int check_csr_host(const ptap_csr* M, bool need_val);

// limits of the fast path (classes.cu)
constexpr int kFastMaxA = 32;   // entries of A(I,:)
constexpr int kFastMaxB = 8;    // entries of each P(k,:) it reaches
constexpr int kFastMaxT = kFastMaxA * kFastMaxB;
constexpr int kFastMaxR = 32;   // distinct columns of (A P)(I,:)
constexpr int kFastMaxP = 8;    // entries of P(I,:)
constexpr int kFastSigCap = 8 + kFastMaxR + 8 * kFastMaxR + kFastMaxT + 3 * kFastMaxR + 8;  // 656 bytes
int build_classes(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, cudaStream_t s);

// numeric.cu
int prepare_numeric(ptap_plan* p);
int numeric_owner(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s);
int numeric_atomic(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s);
int check_numeric_inputs(const ptap_plan* p, const ptap_csr* A, const ptap_csr* P);
// fastnum.cu
int build_index_cache(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, cudaStream_t s);
// host.cu
void host_stage_free(ptap_plan* p);
// twostep.cu
int two_step_numeric(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C, cudaStream_t s);
void two_step_free(ptap_plan* p);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Empty hash slot.  Column indices are < ncols <= INT32_MAX, so never equal;
// empty slots also sort after every key.
constexpr int32_t kEmpty = 0x7fffffff;

__host__ __device__ inline uint32_t hash32(uint32_t k) { return k * 0x9E3779B1u; }

__host__ __device__ inline int ilog2_ceil(uint32_t x) {
  int r = 0;
  while ((1u << r) < x) ++r;
  return r;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace ptap
