// Batched numeric products without any device allocation.
//
// Some callers cannot allocate device memory when the products run: solvers
// that reserve their whole device footprint up front in their own pool and
// forbid any later cudaMalloc, and code on latency-critical paths where a
// cudaMalloc/cudaFree pair would add an implicit device synchronisation.  For
// them, ptap_batch_numeric_noalloc runs several numeric products in one
// persistent launch like ptap_batch_numeric, but without a batch object: the
// work counter, the per-problem descriptors and the work queue live in one
// file-scope __device__ array of PTAP_NOALLOC_SCRATCH_BYTES, which every GPU
// that loads this library holds until the process exits.
//
// Host code never uses that array's name as an address (in host code it is
// only a stand-in for the device symbol): once per device, with that device
// current, cudaGetSymbolAddress yields the device address, and all copies and
// clears go there.  Device code names the array directly.
//
// Every call shares the array and it keeps the previous call's contents, so
// each call clears the work counter before its launch; calls whose work
// overlaps on the GPU (different streams, or devices sharing a context) race
// on the array and must be serialised by the caller.
#include <algorithm>
#include <mutex>

#include "owner.cuh"

namespace ptap {

size_t owner_smem_for(int dtype, const Config& c, int max_rows);
int check_numeric_inputs(const ptap_plan* p, const ptap_csr* A, const ptap_csr* P);

namespace {

constexpr size_t kScratchBytes = PTAP_NOALLOC_SCRATCH_BYTES;
constexpr size_t kDescOffset = 256;
constexpr size_t kDescBytes = (size_t)PTAP_NOALLOC_MAX_PROBLEMS * sizeof(NumArgs<double>);
constexpr size_t kItemsOffset = (kDescOffset + kDescBytes + 255) & ~size_t(255);
constexpr size_t kMaxItems = (kScratchBytes - kItemsOffset) / (2 * sizeof(int32_t));
static_assert(kMaxItems >= PTAP_NOALLOC_MAX_ITEMS, "scratch too small for the stated item limit");
static_assert(sizeof(NumArgs<float>) <= sizeof(NumArgs<double>), "descriptor size");

// The scratch array: [0, 256) work counter; descriptors; work items.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device addresses of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_mutex;

// Host staging for the descriptors and the queue (pageable copies return
// once the data is staged, so the buffer is free again on return).
alignas(256) unsigned char g_host_stage[kScratchBytes - kDescOffset];

template <typename V, int G>
__global__ void __launch_bounds__(256) k_noalloc_batch(int32_t nitems, int slots_log2, int CH,
                                                      int max_rows) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int32_t gflag[256 / 4];
  __shared__ int32_t item;
  int32_t* counter = (int32_t*)g_noalloc_scratch;
  const NumArgs<V>* probs = (const NumArgs<V>*)(g_noalloc_scratch + kDescOffset);
  const int32_t* items = (const int32_t*)(g_noalloc_scratch + kItemsOffset);
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

int scratch_address(unsigned char** out) {
  int dev = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return PTAP_ERR_UNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    PTAP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_addr[dev];
  return PTAP_OK;
}

template <typename V, int G>
int launch(ptap_plan* const* plans, const ptap_csr* A, const ptap_csr* P, void* const* C,
           int32_t count, int64_t nitems, int32_t max_rows, int32_t max_ch, unsigned char* dscratch,
           cudaStream_t s) {
  Config c = plans[0]->cfg;
  c.chunk_entries = max_ch;
  c.block_threads = std::min(c.block_threads, 256);  // the kernel's bound
  // The general owner kernel keeps column indices beside each accumulated
  // value, so plans built for the class-program kernels (chunks of up to
  // 49152 entries) can ask for more shared memory than a CTA may have.  The
  // on-chip capacity is then lowered to what fits: chunks with more entries
  // than that take the kernel's heavy path, which accumulates in C itself
  // with atomics (same result, slower).  Settled before anything is staged.
  int dev = 0, optin = 0;
  PTAP_CUDA(cudaGetDevice(&dev));
  PTAP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  PTAP_CUDA(cudaFuncGetAttributes(&fa, k_noalloc_batch<V, G>));
  optin -= (int)fa.sharedSizeBytes;  // the kernel's static shared memory counts against the limit
  {
    Config c0 = c;
    c0.chunk_entries = 0;
    const size_t fixed = owner_smem_for(plans[0]->dtype, c0, max_rows);
    if (fixed + 64 * (sizeof(V) + sizeof(int32_t)) > (size_t)optin) return PTAP_ERR_UNSUPPORTED;
    const int64_t fit = ((int64_t)optin - (int64_t)fixed) / (int64_t)(sizeof(V) + sizeof(int32_t));
    c.chunk_entries = (int)std::max<int64_t>(64, std::min<int64_t>(c.chunk_entries, fit & ~int64_t(63)));
  }
  const size_t smem = owner_smem_for(plans[0]->dtype, c, max_rows);
  PTAP_TRY(grow_smem_limit((const void*)k_noalloc_batch<V, G>, (int)smem));
  int per_sm = 0;
  PTAP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noalloc_batch<V, G>,
                                                          c.block_threads, smem));
  if (per_sm < 1) return PTAP_ERR_UNSUPPORTED;
  NumArgs<V>* desc = (NumArgs<V>*)g_host_stage;
  int32_t* items = (int32_t*)(g_host_stage + (kItemsOffset - kDescOffset));
  int64_t t = 0;
  for (int32_t q = 0; q < count; ++q) {
    ptap_plan* p = plans[q];
    NumArgs<V>& a = desc[q];
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
    a.max_rows = max_rows;
    a.status = p->status;
    for (int32_t ch = 0; ch < p->nchunks; ++ch) {
      items[2 * t] = q;
      items[2 * t + 1] = ch;
      ++t;
    }
  }
  // the counter must start at zero: the array keeps the previous call's value
  PTAP_CUDA(cudaMemsetAsync(dscratch, 0, kDescOffset, s));
  PTAP_CUDA(cudaMemcpyAsync(dscratch + kDescOffset, desc, (size_t)count * sizeof(NumArgs<V>),
                            cudaMemcpyHostToDevice, s));
  if (nitems > 0)
    PTAP_CUDA(cudaMemcpyAsync(dscratch + kItemsOffset, items, (size_t)nitems * 2 * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s));
  if (nitems == 0) return PTAP_OK;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nitems, (int64_t)num_sms() * per_sm));
  const int slots_log2 = c.force_spill ? 2 : ilog2_ceil((uint32_t)std::max(4, c.ap_slots));
  k_noalloc_batch<V, G><<<grid, c.block_threads, smem, s>>>((int32_t)nitems, slots_log2,
                                                            c.chunk_entries, max_rows);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

}  // namespace

}  // namespace ptap

extern "C" int ptap_batch_numeric_noalloc(ptap_plan* const* plans, const ptap_csr* A,
                                          const ptap_csr* P, void* const* C_vals, int32_t count,
                                          void* stream) {
  ptap::Range range("ptap_batch_numeric_noalloc");
  using namespace ptap;
  if (!plans || !A || !P || !C_vals || count <= 0) return PTAP_ERR_INVALID;
  if (count > PTAP_NOALLOC_MAX_PROBLEMS) return PTAP_ERR_OVERFLOW;
  const ptap_plan* p0 = plans[0];
  if (!p0) return PTAP_ERR_INVALID;
  int64_t nitems = 0;
  int32_t max_rows = 1, max_ch = 64;
  for (int32_t q = 0; q < count; ++q) {
    const ptap_plan* p = plans[q];
    if (!p || p->kind != 0 || p->dtype != p0->dtype) return PTAP_ERR_INVALID;
    if (p->compact) return PTAP_ERR_UNSUPPORTED;  // the general owner kernel takes row ranges
    // one kernel instance serves every plan: the lanes per fine row and the hash
    // slots are compiled into it (chunk sizes and CTA sizes may differ)
    if (p->cfg.group_lanes != p0->cfg.group_lanes || p->cfg.ap_slots != p0->cfg.ap_slots ||
        p->cfg.force_spill != p0->cfg.force_spill)
      return PTAP_ERR_INVALID;
    max_ch = std::max(max_ch, p->cfg.chunk_entries);
    PTAP_TRY(check_numeric_inputs(p, &A[q], &P[q]));
    if (p->nnz_c > 0 && !C_vals[q]) return PTAP_ERR_INVALID;
    nitems += p->nchunks;
    max_rows = std::max(max_rows, p->max_chunk_rows);
  }
  if (nitems > PTAP_NOALLOC_MAX_ITEMS) return PTAP_ERR_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  // The descriptors and the queue are copied from a process-wide host buffer
  // that the next call overwrites; a captured copy would read it at replay,
  // with another call's contents.  So this call is refused during capture.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  PTAP_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return PTAP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  unsigned char* dscratch = nullptr;
  PTAP_TRY(scratch_address(&dscratch));
  const int g = p0->cfg.group_lanes;
  if (p0->dtype == PTAP_F64) {
    if (g == 4) return launch<double, 4>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
    if (g == 8) return launch<double, 8>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
    if (g == 16) return launch<double, 16>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
    if (g == 32) return launch<double, 32>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
  } else {
    if (g == 4) return launch<float, 4>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
    if (g == 8) return launch<float, 8>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
    if (g == 16) return launch<float, 16>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
    if (g == 32) return launch<float, 32>(plans, A, P, C_vals, count, nitems, max_rows, max_ch, dscratch, s);
  }
  return PTAP_ERR_INVALID;
}
