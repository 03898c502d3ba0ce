// iwf_apply_host: H~ psi for a block held in host memory, with the host-to-device copies,
// the apply and the device-to-host copies of successive chunks of vectors overlapped on three
// streams. Only host-side orchestration lives here; the arithmetic is apply_impl's.
#include <algorithm>
#include <cstdint>
#include <string>

#include "common.cuh"

namespace iwf {

namespace {

enum { kH2D = 0, kCompute = 1, kD2H = 2 };
// events: 0 start; per slot s in {0, 1}: 1 + s input ready, 3 + s input free, 5 + s output
// ready, 7 + s output free
constexpr int kEvStart = 0;
int ev_in_ready(int s) { return 1 + s; }
int ev_in_free(int s) { return 3 + s; }
int ev_out_ready(int s) { return 5 + s; }
int ev_out_free(int s) { return 7 + s; }

iwf_status ensure_pipeline(iwf_plan* p, size_t chunk_bytes) {
  for (int i = 0; i < 3; ++i)
    if (!p->host_stream[i])
      IWF_CUDA(cudaStreamCreateWithFlags(&p->host_stream[i], cudaStreamNonBlocking));
  for (int i = 0; i < 9; ++i)
    if (!p->host_ev[i]) IWF_CUDA(cudaEventCreateWithFlags(&p->host_ev[i], cudaEventDisableTiming));
  if (p->host_chunk_bytes >= chunk_bytes) return IWF_OK;
  for (int s = 0; s < 2; ++s) {
    cudaFree(p->d_hin[s]);
    cudaFree(p->d_hout[s]);
    p->d_hin[s] = p->d_hout[s] = nullptr;
  }
  p->host_chunk_bytes = 0;
  for (int s = 0; s < 2; ++s) {
    if (cudaMalloc(&p->d_hin[s], chunk_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_hout[s], chunk_bytes) != cudaSuccess)
      return fail(IWF_ERR_ALLOC, "iwf_apply_host: staging buffers");
  }
  p->host_chunk_bytes = chunk_bytes;
  return IWF_OK;
}

}  // namespace

void release_host_pipeline(iwf_plan* p) {
  for (int s = 0; s < 2; ++s) {
    cudaFree(p->d_hin[s]);
    cudaFree(p->d_hout[s]);
    p->d_hin[s] = p->d_hout[s] = nullptr;
  }
  p->host_chunk_bytes = 0;
  for (int i = 0; i < 9; ++i)
    if (p->host_ev[i]) { cudaEventDestroy(p->host_ev[i]); p->host_ev[i] = nullptr; }
  for (int i = 0; i < 3; ++i)
    if (p->host_stream[i]) { cudaStreamDestroy(p->host_stream[i]); p->host_stream[i] = nullptr; }
}

iwf_status apply_host_impl(iwf_plan* p, int precision, const void* psi_host, void* hpsi_host,
                           int nvec, cudaStream_t stream) {
  if (nvec < 0) return fail(IWF_ERR_ARG, "iwf_apply_host: nvec < 0");
  if (nvec == 0) return IWF_OK;
  if (!psi_host || !hpsi_host) return fail(IWF_ERR_ARG, "iwf_apply_host: null host pointer");
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_apply_host: unknown precision");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_apply_host: no potential set");
  const size_t vbytes = (size_t)p->g.N * (precision == IWF_PREC_F64 ? 16 : 8);
  const uintptr_t a = reinterpret_cast<uintptr_t>(psi_host), b = reinterpret_cast<uintptr_t>(hpsi_host);
  const uintptr_t total = (uintptr_t)vbytes * nvec;
  if (a < b + total && b < a + total) return fail(IWF_ERR_ARG, "iwf_apply_host: psi and hpsi overlap");
  // chunk: at most the apply's L2 chunk, and at least four chunks per block so that copies
  // in both directions overlap the compute
  const int ti = precision == IWF_PREC_F64 ? 0 : 1;
  int cv = (int)(((size_t)p->tune_chunk_mb[ti] << 20) / vbytes);
  cv = std::max(1, std::min(cv, (nvec + 3) / 4));
  IWF_TRY(ensure_pipeline(p, (size_t)cv * vbytes));
  cudaStream_t* hs = p->host_stream;
  cudaEvent_t* ev = p->host_ev;
  IWF_CUDA(cudaEventRecord(ev[kEvStart], stream));
  for (int i = 0; i < 3; ++i) IWF_CUDA(cudaStreamWaitEvent(hs[i], ev[kEvStart], 0));
  const char* hin = static_cast<const char*>(psi_host);
  char* hout = static_cast<char*>(hpsi_host);
  const int nchunks = (nvec + cv - 1) / cv;
  for (int k = 0; k < nchunks; ++k) {
    const int s = k & 1;
    const size_t off = (size_t)k * cv * vbytes;
    const int nv = std::min(cv, nvec - k * cv);
    const size_t bytes = (size_t)nv * vbytes;
    // host -> device, once the apply of chunk k - 2 has finished reading this input buffer
    if (k >= 2) IWF_CUDA(cudaStreamWaitEvent(hs[kH2D], ev[ev_in_free(s)], 0));
    IWF_CUDA(cudaMemcpyAsync(p->d_hin[s], hin + off, bytes, cudaMemcpyHostToDevice, hs[kH2D]));
    IWF_CUDA(cudaEventRecord(ev[ev_in_ready(s)], hs[kH2D]));
    // apply, once the input has arrived and chunk k - 2's result has left this output buffer
    IWF_CUDA(cudaStreamWaitEvent(hs[kCompute], ev[ev_in_ready(s)], 0));
    if (k >= 2) IWF_CUDA(cudaStreamWaitEvent(hs[kCompute], ev[ev_out_free(s)], 0));
    IWF_TRY(apply_impl(p, precision, p->d_hin[s], p->d_hout[s], nv, hs[kCompute]));
    IWF_CUDA(cudaEventRecord(ev[ev_in_free(s)], hs[kCompute]));
    IWF_CUDA(cudaEventRecord(ev[ev_out_ready(s)], hs[kCompute]));
    // device -> host
    IWF_CUDA(cudaStreamWaitEvent(hs[kD2H], ev[ev_out_ready(s)], 0));
    IWF_CUDA(cudaMemcpyAsync(hout + off, p->d_hout[s], bytes, cudaMemcpyDeviceToHost, hs[kD2H]));
    IWF_CUDA(cudaEventRecord(ev[ev_out_free(s)], hs[kD2H]));
  }
  // the caller's stream continues after the last copy back; the call returns when it is done
  IWF_CUDA(cudaStreamWaitEvent(stream, ev[ev_out_free((nchunks - 1) & 1)], 0));
  // synchronises `stream` and reports a pipelined pass that gave up waiting
  return check_apply_error(p, stream);
}

}  // namespace iwf
