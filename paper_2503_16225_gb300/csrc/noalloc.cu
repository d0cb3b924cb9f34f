// Allocation-free overlap entry point.
//
// eacg_overlap_noalloc computes the same block overlaps A_k^* B_k as the library's Gram
// kernels, for callers that cannot allocate device memory themselves: code running inside
// a memory pool that forbids cudaMalloc, or a host process whose device allocations are all
// owned by another runtime that would not see (or would fail) a cudaMalloc of ours.  Its one piece
// of scratch (the partial sums of the split reduction) is a fixed array in this file's
// device memory, so the call itself never allocates.  Every GPU that loads the library
// holds that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/eacg.h"
#include "kernels.h"

namespace {

// Partial sums of the split reduction (K * ceil(n / 1024) * p * p complex values).
static __device__ __align__(256) double2 g_overlap_scratch[EACG_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_overlap_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" eacg_status eacg_overlap_noalloc(int K, int n, int p, const double* a_dev, const double* b_dev,
                                            double* c_dev, void* stream) {
  if (K < 1 || n < 1 || p < 1 || !a_dev || !b_dev || !c_dev) return EACG_EINVAL;
  if (K > 65535) return EACG_EINVAL;  // the kernels take one grid row (z or y) per k-point
  if (eacg::dense_cn_work(K, n, p, p) > (size_t)EACG_NOALLOC_MAX_PARTIALS) return EACG_EINVAL;
  void* work = nullptr;
  if (scratch_address(&work) != cudaSuccess) {
    cudaGetLastError();
    return EACG_ECUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  // every partial the reduction reads is written by the same call first, so the
  // scratch needs no clearing between calls
  eacg::dense_gemm_cn(K, n, p, p, reinterpret_cast<const double2*>(a_dev), (size_t)p * n, n,
                      reinterpret_cast<const double2*>(b_dev), (size_t)p * n, n, reinterpret_cast<double2*>(c_dev),
                      (size_t)p * p, p, one, zero, reinterpret_cast<double2*>(work), nullptr, st);
  if (cudaGetLastError() != cudaSuccess) return EACG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return EACG_ECUDA;
  return EACG_OK;
}
