// Value movement of the row-partitioned product (Section 2, Eq. 1-3; Alg. 7-8).
//
// With the fine rows split into blocks, one per process, a process needs the
// rows of P that its block of A references but another process owns (P~_r,
// gathered by one sparse exchange per phase), and it produces outer-product
// contributions to coarse rows that other processes own (C_s, sent to their
// owners, who add them).  The patterns of both exchanges are fixed by the
// symbolic phase; each numeric phase moves values only.  These two kernels are
// that movement: packing values into a send buffer by a fixed index list, and
// adding received (or local) values into C at fixed positions.
#include "common.cuh"

namespace ptap {
namespace {

template <typename V>
__global__ void k_gather(const V* __restrict__ src, const int32_t* __restrict__ idx, int64_t n,
                         V* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = src[idx[e]];
}

// dst[dst_idx[e]] += src[src_idx ? src_idx[e] : e]; dst_idx holds distinct
// positions within one call, so no two threads touch one entry.
template <typename V>
__global__ void k_scatter_add(const V* __restrict__ src, const int32_t* __restrict__ src_idx,
                              const int32_t* __restrict__ dst_idx, int64_t n, V* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[dst_idx[e]] += src[src_idx ? src_idx[e] : e];
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), num_sms() * 8)); }

}  // namespace
}  // namespace ptap

extern "C" int ptap_gather(const void* src, const int32_t* src_idx, int64_t n, int32_t dtype, void* out,
                           void* stream) {
  if (n < 0 || (dtype != PTAP_F64 && dtype != PTAP_F32)) return PTAP_ERR_INVALID;
  if (n == 0) return PTAP_OK;
  if (!src || !src_idx || !out) return PTAP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == PTAP_F64)
    ptap::k_gather<double><<<ptap::grid_for(n), 256, 0, s>>>((const double*)src, src_idx, n, (double*)out);
  else
    ptap::k_gather<float><<<ptap::grid_for(n), 256, 0, s>>>((const float*)src, src_idx, n, (float*)out);
  PTAP_LAUNCHED();
  return PTAP_OK;
}

extern "C" int ptap_scatter_add(const void* src, const int32_t* src_idx, const int32_t* dst_idx, int64_t n,
                                int32_t dtype, void* dst, void* stream) {
  if (n < 0 || (dtype != PTAP_F64 && dtype != PTAP_F32)) return PTAP_ERR_INVALID;
  if (n == 0) return PTAP_OK;
  if (!src || !dst_idx || !dst) return PTAP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == PTAP_F64)
    ptap::k_scatter_add<double><<<ptap::grid_for(n), 256, 0, s>>>((const double*)src, src_idx, dst_idx, n,
                                                                   (double*)dst);
  else
    ptap::k_scatter_add<float><<<ptap::grid_for(n), 256, 0, s>>>((const float*)src, src_idx, dst_idx, n,
                                                                  (float*)dst);
  PTAP_LAUNCHED();
  return PTAP_OK;
}
