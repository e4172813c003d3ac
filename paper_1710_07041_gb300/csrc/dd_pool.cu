// Cache of solver workspaces. An FGMRES(16) solve on 64x32^3 holds about
// 11 GB of device buffers (the double-float Krylov basis, the preconditioned
// vectors, the solution and scratch fields) and a few pinned host buffers;
// allocating and freeing them on every dd_solve call costs milliseconds of
// host time in which the GPU idles (cudaFree also synchronises the device).
// Buffers a solver releases are kept here, keyed by (device, size), and
// handed to the next solver that asks for the same size. The cache is
// bounded (half the device memory, 64 MB of pinned host memory); a device
// allocation that fails releases the cache and is tried once more, and
// dd_release_workspace() gives everything back.
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "dd_internal.cuh"
#include "dd_pool.cuh"

namespace dd {

namespace {

struct Pool {
  std::mutex mu;
  std::multimap<std::pair<int, size_t>, void *> dev;    // (device, bytes) -> buffer
  std::multimap<std::pair<int, size_t>, void *> host;   // pinned host buffers
  std::map<int, size_t> dev_bytes;                      // cached device bytes per device
  size_t host_bytes = 0;
};

Pool &pool() {
  static Pool *p = new Pool;   // never destroyed: no CUDA call runs at process exit
  return *p;
}

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

void *take(std::multimap<std::pair<int, size_t>, void *> &m, int dev, size_t n) {
  auto it = m.find({dev, n});
  if (it == m.end()) return nullptr;
  void *p = it->second;
  m.erase(it);
  return p;
}

constexpr size_t HOST_CAP = 64u << 20;

}  // namespace

void *pool_dev_alloc(size_t n) {
  if (n == 0) return nullptr;
  const int d = current_device();
  Pool &P = pool();
  {
    std::lock_guard<std::mutex> lk(P.mu);
    if (void *p = take(P.dev, d, n)) {
      P.dev_bytes[d] -= n;
      return p;
    }
  }
  void *p = nullptr;
  if (cudaMalloc(&p, n) == cudaSuccess) return p;
  cudaGetLastError();
  pool_release();   // the cached buffers may be what stands in the way
  if (cudaMalloc(&p, n) == cudaSuccess) return p;
  cudaGetLastError();
  return nullptr;
}

void pool_dev_free(void *p, size_t n) {
  if (!p) return;
  const int d = current_device();
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  Pool &P = pool();
  {
    std::lock_guard<std::mutex> lk(P.mu);
    if (P.dev_bytes[d] + n <= total_b / 2) {
      P.dev.emplace(std::make_pair(d, n), p);
      P.dev_bytes[d] += n;
      return;
    }
  }
  cudaFree(p);
}

void *pool_host_alloc(size_t n) {
  if (n == 0) return nullptr;
  const int d = current_device();
  Pool &P = pool();
  {
    std::lock_guard<std::mutex> lk(P.mu);
    if (void *p = take(P.host, d, n)) {
      P.host_bytes -= n;
      return p;
    }
  }
  void *p = nullptr;
  if (cudaMallocHost(&p, n) == cudaSuccess) return p;
  cudaGetLastError();
  return nullptr;
}

void pool_host_free(void *p, size_t n) {
  if (!p) return;
  const int d = current_device();
  Pool &P = pool();
  {
    std::lock_guard<std::mutex> lk(P.mu);
    if (P.host_bytes + n <= HOST_CAP) {
      P.host.emplace(std::make_pair(d, n), p);
      P.host_bytes += n;
      return;
    }
  }
  cudaFreeHost(p);
}

size_t pool_cached_bytes() {
  const int d = current_device();
  Pool &P = pool();
  std::lock_guard<std::mutex> lk(P.mu);
  auto it = P.dev_bytes.find(d);
  return it == P.dev_bytes.end() ? 0 : it->second;
}

void pool_release() {
  Pool &P = pool();
  std::multimap<std::pair<int, size_t>, void *> dev, host;
  {
    std::lock_guard<std::mutex> lk(P.mu);
    dev.swap(P.dev);
    host.swap(P.host);
    P.dev_bytes.clear();
    P.host_bytes = 0;
  }
  int cur = current_device();
  for (auto &e : dev) {
    cudaSetDevice(e.first.first);
    cudaFree(e.second);
  }
  cudaSetDevice(cur);
  for (auto &e : host) cudaFreeHost(e.second);
}

}  // namespace dd

extern "C" int dd_release_workspace(void) {
  dd::pool_release();
  return DD_OK;
}
