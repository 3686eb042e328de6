// te_probe.cu - measurement of the random-gather ceiling that bounds the SpMV
// on graphs with random vertex ids: every non-zero reads one scattered 4-byte
// value of x, so the SpMV can go no faster than the GPU serves such reads.
// The probe times random reads of a device table (indices from an integer
// hash of the thread and iteration, reduced modulo the table size, so every
// read is in bounds) with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "te_common.cuh"
#include "te_internal.h"
#include "topk_eigs.h"

namespace te {

TE_DEV uint32_t probe_hash(uint32_t v) {  // an integer mixing function
  v ^= v >> 16;
  v *= 0x7feb352dU;
  v ^= v >> 15;
  v *= 0x846ca68bU;
  v ^= v >> 16;
  return v;
}

__global__ void gather_probe_kernel(const float* __restrict__ x, uint32_t n, int iters,
                                    float* out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  for (int it = 0; it < iters; ++it) {
    uint32_t idx[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) idx[u] = probe_hash(t * 8191u + it * 131071u + u * 524287u) % n;
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(x + idx[u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  out[t] = acc;  // keeps the reads live
}

}  // namespace te

extern "C" te_status te_probe_gather(int64_t table_elems, void* stream, double* gathers_per_s) {
  using namespace te;
  if (!gathers_per_s || table_elems < 1024 || table_elems > ((int64_t)1 << 31)) {
    set_last_error("te_probe_gather: table_elems must be in [1024, 2^31]");
    return TE_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 256, grid = sms * 8, iters = 64;
  float* buf = nullptr;
  if (e == cudaSuccess)
    e = cudaMalloc(&buf, sizeof(float) * ((size_t)table_elems + (size_t)grid * block));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(float) * (size_t)table_elems, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      gather_probe_kernel<<<grid, block, 0, s>>>(buf, (uint32_t)table_elems, iters,
                                                 buf + table_elems);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) {
    set_last_error(std::string("te_probe_gather: ") + cudaGetErrorString(e));
    return TE_ERR_CUDA;
  }
  *gathers_per_s = (double)grid * block * iters * 8 / (best * 1e-3);
  return TE_OK;
}
