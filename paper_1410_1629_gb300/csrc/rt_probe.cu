// rt_probe_bandwidth: the read bandwidth this GPU sustains from a buffer of a
// given size, measured with the library's own kernel (the denominator of
// roofline fractions for kernels whose working set stays in L2, for which no
// vendor figure is used).  Not part of the transport method.
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace {

// Every thread sums float4 loads over a grid-stride loop, `passes` times
// over the whole buffer; the sum is written only if it equals a value no
// input produces, so the loads cannot be removed.
__global__ void __launch_bounds__(512) k_read(const float4* __restrict__ buf, size_t n4, int passes,
                                              float* __restrict__ sink) {
  float acc = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(&buf[i]);  // cached in L2 only: the L1 does not serve repeats
      acc += (v.x + v.y) + (v.z + v.w);
    }
  }
  if (acc == -1.0f) *sink = acc;
}

__global__ void k_fill(float4* buf, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x)
    buf[i] = make_float4(1.0f, 2.0f, 3.0f, 4.0f);
}

}  // namespace

extern "C" rt_status rt_probe_bandwidth(int32_t device, uint64_t bytes, int32_t passes, int32_t repeats,
                                        double* gb_per_s) {
  if (!gb_per_s || bytes < 4096 || passes < 1 || repeats < 1) {
    rtk::set_context_free_error("rt_probe_bandwidth: bad arguments");
    return RT_ERR_ARG;
  }
  *gb_per_s = 0.0;
  cudaError_t e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  float4* buf = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const size_t n4 = (size_t)(bytes / 16);
  if (e == cudaSuccess) e = cudaMalloc(&buf, n4 * 16);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const unsigned blocks = (unsigned)sms * 4u;
  if (e == cudaSuccess) {
    k_fill<<<blocks, 512>>>(buf, n4);
    k_read<<<blocks, 512>>>(buf, n4, 1, sink);  // warm-up: the buffer's lines reach L2 if they fit
    e = cudaGetLastError();
  }
  float best = -1.0f;
  for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0);
    if (e == cudaSuccess) k_read<<<blocks, 512>>>(buf, n4, passes, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (best < 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    rtk::set_context_free_error(cudaGetErrorString(e));
    return RT_ERR_CUDA;
  }
  *gb_per_s = (double)n4 * 16.0 * passes / (best * 1e-3) / 1e9;
  return RT_OK;
}
