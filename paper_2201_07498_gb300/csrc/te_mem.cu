// te_mem.cu - device memory of plans, layouts and their temporaries.
//
// A plan allocates its work memory, the copy of a host matrix, the row order
// and the layout's scratch when it is created, and frees most of it again
// within the same call or when it is destroyed: about 13 GB per solve for
// R-MAT 2^24 from a host CSR.  Through cudaMalloc / cudaFree every one of
// those calls maps or unmaps pages (≈ 8 ms of a 114 ms end-to-end solve).
// Here they come from a stream-ordered memory pool per device that the
// library owns: freed blocks stay mapped and serve the next plan, up to the
// pool's release threshold (te_set_memory_cache; default: keep everything).
// An allocation that finds the device full first returns what the pool holds
// to the driver and tries once more.  te_release_cached_memory gives back
// every unused block at once.
//
// Semantics are those of cudaMalloc / cudaFree: dev_alloc returns memory that
// every stream may use at once (the allocation runs on an idle stream of the
// library, which is synchronised), and dev_free first waits for the device
// to be idle, as cudaFree does, so that no queued kernel still reads the
// block when the pool hands it out again.
#include <mutex>

#include "te_internal.h"

namespace te {
namespace {

constexpr int MAX_DEVICES = 64;

struct DevPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t s = nullptr;  // the allocations' and frees' stream (kept idle)
};

std::mutex g_mu;
DevPool g_pool[MAX_DEVICES];
uint64_t g_keep = UINT64_MAX;  // release threshold of every pool

cudaError_t pool_of(int dev, DevPool** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  DevPool& d = g_pool[dev];
  if (!d.pool) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    cudaError_t e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = g_keep;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    d.pool = p;
    d.s = s;
  }
  *out = &d;
  return cudaSuccess;
}

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  DevPool* d = nullptr;
  if (e == cudaSuccess) e = pool_of(dev, &d);
  if (e != cudaSuccess) return e;
  if (bytes == 0) bytes = 1;
  e = cudaMallocFromPoolAsync(p, bytes, d->pool, d->s);
  if (e == cudaErrorMemoryAllocation) {
    // the blocks the pool keeps go back to the driver, then once more
    (void)cudaGetLastError();
    e = cudaStreamSynchronize(d->s);
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(d->pool, 0);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, d->pool, d->s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->s);
  if (e != cudaSuccess) *p = nullptr;
  return e;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) return e;
  int cur = 0;
  e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  const int dev = a.device;
  DevPool* d = nullptr;
  e = pool_of(dev, &d);
  if (e != cudaSuccess) return e;
  if (dev != cur) e = cudaSetDevice(dev);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaFreeAsync(p, d->s);
  if (dev != cur) cudaSetDevice(cur);
  return e;
}

cudaError_t dev_free_on(void* p, cudaStream_t s) {
  return p ? cudaFreeAsync(p, s) : cudaSuccess;
}

}  // namespace te

using te::g_keep;
using te::g_mu;
using te::g_pool;

extern "C" {

te_status te_set_memory_cache(uint64_t keep_bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_keep = keep_bytes;
  for (int dev = 0; dev < te::MAX_DEVICES; ++dev) {
    if (!g_pool[dev].pool) continue;
    uint64_t keep = keep_bytes;
    if (cudaMemPoolSetAttribute(g_pool[dev].pool, cudaMemPoolAttrReleaseThreshold, &keep) !=
        cudaSuccess)
      return TE_ERR_CUDA;
  }
  return TE_OK;
}

te_status te_release_cached_memory(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int dev = 0; dev < te::MAX_DEVICES; ++dev) {
    if (!g_pool[dev].pool) continue;
    if (cudaStreamSynchronize(g_pool[dev].s) != cudaSuccess ||
        cudaMemPoolTrimTo(g_pool[dev].pool, 0) != cudaSuccess)
      return TE_ERR_CUDA;
  }
  return TE_OK;
}

te_status te_memory_cached(int32_t device, uint64_t* reserved_bytes, uint64_t* used_bytes) {
  if (!reserved_bytes || !used_bytes || device < 0 || device >= te::MAX_DEVICES)
    return TE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  *reserved_bytes = 0;
  *used_bytes = 0;
  cudaMemPool_t p = g_pool[device].pool;
  if (!p) return TE_OK;
  uint64_t r = 0, u = 0;
  if (cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &r) != cudaSuccess ||
      cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &u) != cudaSuccess)
    return TE_ERR_CUDA;
  *reserved_bytes = r;
  *used_bytes = u;
  return TE_OK;
}

}  // extern "C"
