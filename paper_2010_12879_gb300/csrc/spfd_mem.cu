// Device (and pinned host) memory cache.
//
// A context allocates a few dozen device buffers (4.6 GB for the 2 mm body
// with the mixed-precision copies), and cudaMalloc/cudaFree of that much
// memory takes milliseconds per build.  Blocks a context releases are kept
// in a process-wide cache, one per device, and handed to later contexts
// whose requests they fit.  Only whole idle blocks enter the cache: a
// context returns its blocks in spfd_destroy after synchronising its
// stream, so no queued kernel still uses them.  spfd_release_cached_memory
// gives the cached blocks back to the driver, and a failed cudaMalloc does
// so once before it retries.
#include <map>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "spfd_mem.cuh"

namespace spfd {

namespace {

struct Cache {
  std::mutex mu;
  std::vector<std::multimap<size_t, void *>> free_by_device;  // block size -> block
  std::multimap<size_t, void *> free_host;                    // pinned host blocks
  size_t held = 0;                                            // bytes in the cache
};

Cache &cache() {
  static Cache *c = new Cache;  // never destroyed: may be used during exit
  return *c;
}

// Requests are rounded up so that repeated builds of the same problem hit
// the cache with identical sizes: 512 B below 1 MiB, 2 MiB above.
size_t round_up(size_t bytes) {
  const size_t g = bytes < (1u << 20) ? 512 : (2u << 20);
  return (bytes + g - 1) / g * g;
}

}  // namespace

cudaError_t mem_get(int device, size_t bytes, void **p, size_t *block) {
  const size_t want = round_up(bytes < 1 ? 1 : bytes);
  Cache &c = cache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    if ((size_t)device < c.free_by_device.size()) {
      auto &m = c.free_by_device[device];
      auto it = m.lower_bound(want);
      // take a block at most 25 % (and at least 2 MiB) larger than asked
      const size_t slack = want / 4 > (2u << 20) ? want / 4 : (2u << 20);
      if (it != m.end() && it->first <= want + slack) {
        *p = it->second;
        *block = it->first;
        c.held -= it->first;
        m.erase(it);
        return cudaSuccess;
      }
    }
  }
  cudaError_t e = cudaMalloc(p, want);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    mem_release_all();
    e = cudaMalloc(p, want);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  *block = want;
  return cudaSuccess;
}

void mem_put(int device, void *p, size_t block) {
  if (!p) return;
  Cache &c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  if ((size_t)device >= c.free_by_device.size()) c.free_by_device.resize(device + 1);
  c.free_by_device[device].emplace(block, p);
  c.held += block;
}

cudaError_t host_get(size_t bytes, void **p, size_t *block) {
  const size_t want = round_up(bytes < 1 ? 1 : bytes);
  Cache &c = cache();
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.free_host.lower_bound(want);
    if (it != c.free_host.end() && it->first <= 2 * want + (1u << 20)) {
      *p = it->second;
      *block = it->first;
      c.held -= it->first;
      c.free_host.erase(it);
      return cudaSuccess;
    }
  }
  cudaError_t e = cudaMallocHost(p, want);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  *block = want;
  return cudaSuccess;
}

void host_put(void *p, size_t block) {
  if (!p) return;
  Cache &c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  c.free_host.emplace(block, p);
  c.held += block;
}

size_t mem_release_all() {
  Cache &c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  size_t freed = 0;
  for (auto &kv : c.free_host) {
    cudaFreeHost(kv.second);
    freed += kv.first;
  }
  c.free_host.clear();
  int cur = 0;
  cudaGetDevice(&cur);
  for (size_t d = 0; d < c.free_by_device.size(); ++d) {
    auto &m = c.free_by_device[d];
    if (m.empty()) continue;
    cudaSetDevice((int)d);
    for (auto &kv : m) {
      cudaFree(kv.second);
      freed += kv.first;
    }
    m.clear();
  }
  cudaSetDevice(cur);
  c.held = 0;
  return freed;
}

size_t mem_cached_bytes() {
  Cache &c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  return c.held;
}

}  // namespace spfd
