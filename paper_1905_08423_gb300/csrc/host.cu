// Numeric product from host-resident values: ptap_numeric_host.
//
// The numeric phase is repeated whenever the values of A and P change
// (Section 4.1: one symbolic, many numeric products).  When those values are
// assembled on the host, each product needs them on the device and its
// result back.  This file stages them through plan-owned device buffers,
// double-buffered, with the copies on two internal streams:
//
//   copy-in stream :  H2D A, P values of call k  (into set k % 2)
//   caller stream  :  numeric product k           (after its H2D)
//   copy-out stream:  D2H C values of call k      (after the product)
//   caller stream  :  waits for that D2H, so a synchronised caller stream
//                     means C_val_host is complete
//
// Call k+1's host-to-device copy waits only for the buffers of call k-1 to
// be released (their D2H done), so it runs under product k and its D2H; a
// step then costs about max(H2D, product + D2H) instead of their sum.  The
// product itself is ptap_numeric on the staged values: every kernel path
// (class programs, general, atomic, two-step) is available.
#include "common.cuh"

namespace ptap {

struct HostStage {
  void* a[2] = {nullptr, nullptr};
  void* p[2] = {nullptr, nullptr};
  void* c[2] = {nullptr, nullptr};
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_kernel[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr};
  bool out_recorded[2] = {false, false};
  int next = 0;
};

void host_stage_free(ptap_plan* p) {
  HostStage* h = p->host;
  if (!h) return;
  if (h->s_in) cudaStreamSynchronize(h->s_in);
  if (h->s_out) cudaStreamSynchronize(h->s_out);
  for (int b = 0; b < 2; ++b) {
    if (h->ev_in[b]) cudaEventDestroy(h->ev_in[b]);
    if (h->ev_kernel[b]) cudaEventDestroy(h->ev_kernel[b]);
    if (h->ev_out[b]) cudaEventDestroy(h->ev_out[b]);
  }
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  delete h;  // the buffers belong to the plan's allocator and go with it
  p->host = nullptr;
}

static int host_stage_init(ptap_plan* p) {
  if (p->host) return PTAP_OK;
  HostStage* h = new (std::nothrow) HostStage();
  if (!h) return PTAP_ERR_OOM;
  p->host = h;
  const size_t vb = p->dtype == PTAP_F64 ? 8 : 4;
  for (int b = 0; b < 2; ++b) {
    PTAP_TRY(p->mem.get(&h->a[b], (size_t)p->nnz_a * vb));
    PTAP_TRY(p->mem.get(&h->p[b], (size_t)p->nnz_p * vb));
    PTAP_TRY(p->mem.get(&h->c[b], (size_t)p->nnz_c * vb));
    PTAP_CUDA(cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming));
    PTAP_CUDA(cudaEventCreateWithFlags(&h->ev_kernel[b], cudaEventDisableTiming));
    PTAP_CUDA(cudaEventCreateWithFlags(&h->ev_out[b], cudaEventDisableTiming));
  }
  PTAP_CUDA(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
  PTAP_CUDA(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
  // the allocations above were made on the plan's stream
  PTAP_CUDA(cudaStreamSynchronize(p->stream));
  return PTAP_OK;
}

}  // namespace ptap

extern "C" int ptap_numeric(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, void* C_val, void* stream);

extern "C" int ptap_numeric_host(ptap_plan* p, const ptap_csr* A, const ptap_csr* P, const void* A_val_host,
                                 const void* P_val_host, void* C_val_host, void* stream) {
  ptap::Range range("ptap_numeric_host");
  if (!p || !A || !P) return PTAP_ERR_INVALID;
  if ((p->nnz_a > 0 && !A_val_host) || (p->nnz_p > 0 && !P_val_host) || (p->nnz_c > 0 && !C_val_host))
    return PTAP_ERR_INVALID;
  ptap_csr Ad = *A, Pd = *P;
  Ad.val = Pd.val = reinterpret_cast<const void*>(1);  // placeholders: checked for presence only
  PTAP_TRY(ptap::check_numeric_inputs(p, &Ad, &Pd));
  PTAP_TRY(ptap::host_stage_init(p));
  ptap::HostStage* h = p->host;
  cudaStream_t s = (cudaStream_t)stream;
  const int b = h->next;
  h->next ^= 1;
  const size_t vb = p->dtype == PTAP_F64 ? 8 : 4;
  // inputs: wait until set b's previous product has been copied out
  if (h->out_recorded[b]) PTAP_CUDA(cudaStreamWaitEvent(h->s_in, h->ev_out[b], 0));
  if (p->nnz_a > 0)
    PTAP_CUDA(cudaMemcpyAsync(h->a[b], A_val_host, (size_t)p->nnz_a * vb, cudaMemcpyHostToDevice, h->s_in));
  if (p->nnz_p > 0)
    PTAP_CUDA(cudaMemcpyAsync(h->p[b], P_val_host, (size_t)p->nnz_p * vb, cudaMemcpyHostToDevice, h->s_in));
  PTAP_CUDA(cudaEventRecord(h->ev_in[b], h->s_in));
  // the product on the caller's stream
  PTAP_CUDA(cudaStreamWaitEvent(s, h->ev_in[b], 0));
  Ad.val = h->a[b];
  Pd.val = h->p[b];
  PTAP_TRY(ptap_numeric(p, &Ad, &Pd, h->c[b], stream));
  PTAP_CUDA(cudaEventRecord(h->ev_kernel[b], s));
  // result back to the host; the caller's stream waits for it
  PTAP_CUDA(cudaStreamWaitEvent(h->s_out, h->ev_kernel[b], 0));
  if (p->nnz_c > 0)
    PTAP_CUDA(cudaMemcpyAsync(C_val_host, h->c[b], (size_t)p->nnz_c * vb, cudaMemcpyDeviceToHost, h->s_out));
  PTAP_CUDA(cudaEventRecord(h->ev_out[b], h->s_out));
  h->out_recorded[b] = true;
  PTAP_CUDA(cudaStreamWaitEvent(s, h->ev_out[b], 0));
  return PTAP_OK;
}
