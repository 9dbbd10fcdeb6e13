// Device memory of the library's buffers: one stream-ordered memory pool per device.
//
// Every buffer (DBuf) is allocated with cudaMallocFromPoolAsync and returned with cudaFreeAsync on
// the stream of the entry point that owns it (StreamScope), so that
//  * a free never waits for the device (cudaFree synchronises the whole device and unmaps memory, and
//    a solve allocates and frees its Krylov bases, operand blocks and scratch many times), and
//  * the pool keeps what it has reserved (release threshold: unlimited), so that a context created
//    after another one was freed reuses its device pages instead of mapping new ones.
// The pool is the library's own (not the device's default pool), so the caller's allocators are not
// affected. gfcc_release_cached_memory() gives the unused reserve back to the device.
#include "gfcc_internal.cuh"

#include <cstdint>
#include <mutex>

namespace gfcc {
namespace {

constexpr int kMaxDev = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDev] = {};
thread_local cudaStream_t t_stream = nullptr;

cudaMemPool_t pool_for(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;   // keep freed memory reserved for the next allocations
    if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    g_pool[dev] = p;
  }
  return g_pool[dev];
}

}  // namespace

cudaStream_t current_alloc_stream() { return t_stream; }

StreamScope::StreamScope(cudaStream_t s) : prev(t_stream) { t_stream = s; }
StreamScope::~StreamScope() { t_stream = prev; }

cudaError_t pool_alloc(void** p, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  cudaMemPool_t pool = pool_for(dev);
  if (!pool) return cudaMalloc(p, bytes);   // no pool on this device: plain allocations
  e = cudaMallocFromPoolAsync(p, bytes, pool, t_stream);
  if (e == cudaErrorMemoryAllocation) {
    // the reserve may be held by frees still in flight or fragmented: wait for them, give the unused
    // reserve back to the device and try once more
    cudaGetLastError();
    if (cudaDeviceSynchronize() != cudaSuccess) return cudaGetLastError();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, pool, t_stream);
  }
  return e;
}

void pool_free(void* p) {
  if (!p) return;
  cudaPointerAttributes at;
  bool pooled = false;
  int dev = 0;
  if (cudaPointerGetAttributes(&at, p) == cudaSuccess) {
    dev = at.device;
    if (dev >= 0 && dev < kMaxDev) {
      std::lock_guard<std::mutex> lk(g_pool_mu);
      pooled = g_pool[dev] != nullptr;
    }
  } else {
    cudaGetLastError();
  }
  if (pooled) {
    if (cudaFreeAsync(p, t_stream) != cudaSuccess) cudaGetLastError();
  } else if (cudaFree(p) != cudaSuccess) {
    cudaGetLastError();
  }
}

size_t device_free_bytes() {
  size_t freeb = 0, totalb = 0;
  if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return freeb;
  }
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    pool = g_pool[dev];
  }
  if (!pool) return freeb;
  uint64_t reserved = 0, used = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
    cudaGetLastError();
    return freeb;
  }
  return freeb + (reserved > used ? (size_t)(reserved - used) : 0);
}

}  // namespace gfcc

extern "C" int gfcc_release_cached_memory(void) {
  int rc = GFCC_OK;
  for (int dev = 0; dev < gfcc::kMaxDev; ++dev) {
    cudaMemPool_t pool = nullptr;
    {
      std::lock_guard<std::mutex> lk(gfcc::g_pool_mu);
      pool = gfcc::g_pool[dev];
    }
    if (!pool) continue;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
      cudaGetLastError();
      rc = GFCC_ERR_CUDA;
    }
    cudaSetDevice(cur);
  }
  return rc;
}
