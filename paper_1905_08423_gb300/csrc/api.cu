// Plan management, configuration and error reporting of the C ABI.
#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"

namespace ptap {

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("PTAP_VERBOSE"))
    fprintf(stderr, "ptap: CUDA error %s (%s) in %s at %s:%d\n", cudaGetErrorName(e),
            cudaGetErrorString(e), what, file, line);
}

bool profile_enabled() {
  static const bool on = getenv("PTAP_PROFILE") != nullptr;
  return on;
}

void profile_report(const char* name, double ms) { fprintf(stderr, "ptap: %-44s %9.3f ms\n", name, ms); }

int grow_smem_limit(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limits;  // (device, kernel) -> limit set
  int dev = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limits[{dev, fn}];
  if (bytes <= cur) return PTAP_OK;
  PTAP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  cur = bytes;
  return PTAP_OK;
}

static int pick(int v, int dflt) { return v > 0 ? v : dflt; }

Config resolve_config(const ptap_config* c) {
  Config r;
  if (!c) return r;
  if (c->mode == PTAP_MODE_OWNER || c->mode == PTAP_MODE_ATOMIC) r.mode = c->mode;
  r.chunk_entries = c->chunk_entries > 0 ? std::min(std::max(c->chunk_entries, 64), 65536) : 0;
  r.class_programs = c->class_programs >= 0 ? 1 : 0;
  r.visit_block_log2 = (c->visit_block_log2 > 0 && c->visit_block_log2 <= 24) ? c->visit_block_log2 : 0;
  r.jit = c->specialize > 0 ? 1 : 0;
  if (c->specialize > 0) r.jit_max_classes = std::min(c->specialize, 256);
  r.jit_scope = c->specialize_scope == 1 ? 1 : 0;
  r.jit_async = c->specialize_async != 0 ? 1 : 0;
  const int bt = pick(c->block_threads, r.block_threads);
  r.block_threads = (bt == 64 || bt == 128 || bt == 256 || bt == 512 || bt == 1024) ? bt : r.block_threads;
  const int g = pick(c->group_lanes, r.group_lanes);
  r.group_lanes = (g == 4 || g == 8 || g == 16 || g == 32) ? g : r.group_lanes;
  r.ap_slots = std::min(std::max(pick(c->ap_slots, r.ap_slots), 4), 1024);
  r.debug_checks = c->debug_checks != 0;
  r.cache_indices = c->cache_indices >= 2 ? 2 : c->cache_indices > 0 ? 1 : 0;
  r.general_kernel = c->general_kernel == 1 ? 1 : 0;
  r.compact_chunks = std::max(0, std::min(c->compact_chunks, 4096));
  r.force_spill = c->force_spill != 0;
  return r;
}

}  // namespace ptap

extern "C" {

int ptap_plan_pattern(const ptap_plan* p, int32_t* m, int64_t* nnz, const int32_t** row_ptr,
                      const int32_t** col_idx) {
  if (!p) return PTAP_ERR_INVALID;
  if (m) *m = p->m;
  if (nnz) *nnz = p->nnz_c;
  if (row_ptr) *row_ptr = p->c_rp;
  if (col_idx) *col_idx = p->c_ci;
  return PTAP_OK;
}

int ptap_plan_stats(const ptap_plan* p, ptap_stats* o) {
  if (!p || !o) return PTAP_ERR_INVALID;
  memset(o, 0, sizeof(*o));
  o->n = p->n;
  o->m = p->m;
  o->nnz_a = p->nnz_a;
  o->nnz_p = p->nnz_p;
  o->nnz_c = p->nnz_c;
  o->plan_bytes = p->mem.live;
  o->peak_bytes = p->mem.peak;
  o->symbolic_peak_bytes = p->symbolic_peak;
  o->n_chunks = p->nchunks;
  o->n_heavy_chunks = p->nheavy;
  o->chunk_fine_rows = p->nfrows;
  o->n_spill_rows_symbolic = p->spill_rows;
  o->mode = p->kind == 1 ? 0 : p->cfg.mode;
  o->chunk_entries = p->cfg.chunk_entries;
  o->block_threads = p->cfg.block_threads;
  o->group_lanes = p->cfg.group_lanes;
  o->ap_slots = p->cfg.ap_slots;
  o->kind = p->kind;
  o->fast_path = p->fast;
  o->n_classes = p->nclasses;
  o->n_segments = p->nseg;
  o->n_pieces = (int32_t)std::min<int64_t>(p->npieces, INT32_MAX);
  const bool jit = p->jit_fn.load(std::memory_order_acquire) != nullptr;
  o->n_specialized = jit ? p->jit_classes : 0;
  o->specialized_permille = jit ? (int32_t)(p->jit_coverage * 1000.0 + 0.5) : 0;
  o->specialize_us = (int32_t)std::min(p->jit_ms * 1000.0, 2.0e9);
  o->compact_chunks = p->compact ? 1 : 0;
  o->cache_indices = p->index_mode();
  o->cached_index_bytes = p->rec ? p->rec_bytes + 4 * p->npieces : p->aq ? 4 * p->nnz_a : 0;
  return PTAP_OK;
}

int ptap_plan_check(ptap_plan* p, void* stream) {
  if (!p) return PTAP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t st = 0;
  PTAP_CUDA(cudaStreamSynchronize(s));
  PTAP_CUDA(cudaMemcpy(&st, p->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (st) PTAP_CUDA(cudaMemset(p->status, 0, sizeof(int32_t)));
  return st;
}

void ptap_plan_destroy(ptap_plan* p) {
  if (!p) return;
  if (p->jit_thread) {  // a background compile finishes before the plan goes
    p->jit_thread->join();
    delete p->jit_thread;
    p->jit_thread = nullptr;
  }
  cudaStreamSynchronize(p->stream);
  ptap::host_stage_free(p);
  p->mem.release_all();
  ptap::two_step_free(p);
  delete p;
}

const char* ptap_error_string(int code) {
  switch (code) {
    case PTAP_OK: return "ok";
    case PTAP_ERR_INVALID: return "invalid argument (null pointer, shape, dtype or CSR structure)";
    case PTAP_ERR_PATTERN: return "inputs do not match the pattern the plan was built for";
    case PTAP_ERR_OVERFLOW: return "count does not fit int32 indexing (>= 2^31)";
    case PTAP_ERR_OOM: return "device allocation failed";
    case PTAP_ERR_SPILL: return "device hash table ran out of space";
    case PTAP_ERR_TIMEOUT: return "bounded device wait gave up";
    case PTAP_ERR_CUDA: return "CUDA error";
    case PTAP_ERR_UNSUPPORTED: return "not supported by this build";
  }
  return "unknown error code";
}

int ptap_version(void) { return 100; }

}  // extern "C"
