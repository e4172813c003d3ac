// Launch-configuration autotuner. For each (kernel family, lattice shape,
// precision, right-hand-side count, device) it times every variant once on
// the caller's own buffers (3 runs after a warm-up, CUDA events on the
// caller's stream) and caches the fastest; later calls reuse the choice.
// Tuning synchronises the stream, so it is skipped (variant 0 is used) while
// the stream is being captured into a CUDA graph. DD_TUNE=0 in the
// environment disables tuning; DD_TUNE_VARIANT=<k> forces variant k;
// DD_TUNE_VERBOSE=1 prints every variant's time to stderr.
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "dd_tune.cuh"

namespace dd {
namespace {
std::mutex g_mu;
std::map<std::string, int> g_cache;
}  // namespace

std::string tune_key(const char *kind, const Geom &g, int prec, int nrhs) {
  int dev = 0;
  cudaGetDevice(&dev);
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%d|%d,%d,%d,%d|%d,%d,%d,%d|%d|%d", kind, dev, g.L[0], g.L[1], g.L[2], g.L[3], g.bd[0],
           g.bd[1], g.bd[2], g.bd[3], prec, nrhs);
  return buf;
}

int tuned_variant(const std::string &key, int nvariants, const std::function<int(int)> &run, cudaStream_t st,
                  int *chosen) {
  const char *force = getenv("DD_TUNE_VARIANT");
  if (force) {
    int v = atoi(force);
    *chosen = (v >= 0 && v < nvariants) ? v : 0;
    return DD_OK;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *chosen = it->second;
      return DD_OK;
    }
  }
  const char *off = getenv("DD_TUNE");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  // under capture the cached choice (looked up above) or variant 0 is used
  if ((off && off[0] == '0') || cap != cudaStreamCaptureStatusNone || nvariants == 1) {
    *chosen = 0;
    return DD_OK;
  }
  cudaEvent_t e0, e1;
  DD_CUDA(cudaEventCreate(&e0));
  DD_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = 0, rc = DD_OK;
  const char *verbose = getenv("DD_TUNE_VERBOSE");
  std::string report;
  for (int v = 0; v < nvariants && rc == DD_OK; v++) {
    if ((rc = run(v))) break;
    cudaEventRecord(e0, st);
    for (int k = 0; k < 3 && rc == DD_OK; k++) rc = run(v);
    cudaEventRecord(e1, st);
    if (rc) break;
    rc = cuda_fail(cudaEventSynchronize(e1), "tune");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (verbose) report += " v" + std::to_string(v) + "=" + std::to_string(ms / 3) + "ms";
    if (ms < best) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (verbose) fprintf(stderr, "dd tune %s:%s -> v%d\n", key.c_str(), report.c_str(), best_v);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = best_v;
  *chosen = best_v;
  return DD_OK;
}

int tune_lookup(const std::string &key) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(key);
  return it == g_cache.end() ? -1 : it->second;
}

}  // namespace dd
