// Process-wide cache of idle device blocks (spfd_mem.cu).
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

namespace spfd {

// A block of at least `bytes` on `device` (the current device): from the
// cache when one fits, else from cudaMalloc.  *block receives the block's
// real size, which mem_put needs back.
cudaError_t mem_get(int device, size_t bytes, void **p, size_t *block);
// Returns an idle block (no queued work may still use it) to the cache.
void mem_put(int device, void *p, size_t block);
// Pinned host blocks (staging for asynchronous uploads), cached the same way;
// a block may be put back only once no queued copy reads it.
cudaError_t host_get(size_t bytes, void **p, size_t *block);
void host_put(void *p, size_t block);
// Frees every cached block (device and pinned host); returns the bytes.
size_t mem_release_all();
size_t mem_cached_bytes();

}  // namespace spfd
