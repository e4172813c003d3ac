// Cache of solver workspaces (dd_pool.cu): device buffers keyed by (device,
// size) and pinned host buffers. pool_dev_free / pool_host_free require that
// no queued GPU work still uses the buffer.
#pragma once
#include <cstddef>

namespace dd {
void *pool_dev_alloc(size_t bytes);   // a cached buffer of exactly this size, else cudaMalloc
void pool_dev_free(void *p, size_t bytes);
void *pool_host_alloc(size_t bytes);
void pool_host_free(void *p, size_t bytes);
size_t pool_cached_bytes();   // device bytes cached for the current device
void pool_release();          // free every cached buffer
}  // namespace dd
