// Memory for plans, solvers and batches. Device buffers come from a library-owned stream-ordered pool per device
// whose release threshold keeps freed blocks cached, so creating and destroying plans repeatedly (one plan per
// request) reuses memory instead of calling cudaMalloc / cudaFree, each of which synchronises the device; a
// destroy trims the pool back to an eighth of the device's memory (at least 1 GiB: 35 GB on a GB300), so a
// request-sized plan is reused whole while the memory of an exceptionally large one returns to the device. The
// amount kept is the caller's choice (qp_set_memory_cache; 0 returns every freed block at once), and
// qp_memory_pool_stats reports what the pool holds. Small page-locked host mirrors (solver state, a*) come from a
// process-wide cache by size class for the same reason.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "qp_internal.cuh"

namespace qp {

namespace {

std::mutex g_pool_mutex;
cudaMemPool_t g_pools[64] = {};
std::atomic<uint64_t> g_dev_allocs{0};          // device allocations served by the pool (all devices)
std::atomic<int64_t> g_cache_bytes{-1};         // bytes kept cached after a destroy; -1: an eighth of the device

cudaMemPool_t pool_of_current_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) raise(QP_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    CK(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;   // never trim: freed blocks stay with the pool for the next plan
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

std::mutex g_pinned_mutex;
std::map<size_t, std::vector<void*>> g_pinned_free;   // size class -> cached page-locked blocks

size_t size_class(size_t b) {
  size_t c = 256;
  while (c < b) c <<= 1;
  return c;
}

}  // namespace

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool_of_current_device(), s);
  g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
  if (e != cudaSuccess) {
    cudaGetLastError();
    raise(e == cudaErrorMemoryAllocation ? QP_ERR_OOM : QP_ERR_CUDA,
          "device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

void dev_free(void* p) {
  if (p) cudaFreeAsync(p, 0);
}

// After a plan's buffers went back to the pool: keep up to the cache size (default an eighth of the device memory,
// at least 1 GiB) cached for the next plans, return the rest.
void dev_trim() {
  cudaStreamSynchronize(0);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  size_t keep = 0;
  const int64_t want = g_cache_bytes.load();
  if (want >= 0) {
    keep = (size_t)want;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) tot = 0;
    keep = std::max<size_t>((size_t)1 << 30, tot / 8);
  }
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (g_pools[dev]) cudaMemPoolTrimTo(g_pools[dev], keep);
}

void set_cache_bytes(int64_t bytes) {
  g_cache_bytes.store(bytes < 0 ? -1 : bytes);
  dev_trim();
}

void pool_stats(int64_t* reserved, int64_t* used, uint64_t* allocs) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  uint64_t res = 0, use = 0;
  {
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (dev >= 0 && dev < 64 && g_pools[dev]) {
      CK(cudaMemPoolGetAttribute(g_pools[dev], cudaMemPoolAttrReservedMemCurrent, &res));
      CK(cudaMemPoolGetAttribute(g_pools[dev], cudaMemPoolAttrUsedMemCurrent, &use));
    }
  }
  if (reserved) *reserved = (int64_t)res;
  if (used) *used = (int64_t)use;
  if (allocs) *allocs = g_dev_allocs.load(std::memory_order_relaxed);
}

void* pinned_alloc(size_t bytes) {
  const size_t c = size_class(bytes);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mutex);
    auto it = g_pinned_free.find(c);
    if (it != g_pinned_free.end() && !it->second.empty()) {
      void* p = it->second.back();
      it->second.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  CK(cudaMallocHost(&p, c));
  return p;
}

void pinned_free(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pinned_mutex);
  g_pinned_free[size_class(bytes)].push_back(p);
}

}  // namespace qp
