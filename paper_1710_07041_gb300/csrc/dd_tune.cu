// Launch-configuration autotuner. For each (kernel family, lattice shape,
// precision, right-hand-side count, device) it times every variant once on
// the caller's own buffers (3 runs after a warm-up, CUDA events on the
// caller's stream) and caches the fastest; later calls reuse the choice.
// Tuning synchronises the stream, so it is skipped (variant 0 is used) while
// the stream is being captured into a CUDA graph. DD_TUNE=0 in the
// environment disables tuning; DD_TUNE_VARIANT=<k> forces variant k;
// DD_TUNE_VERBOSE=1 prints every variant's time to stderr;
// DD_TUNE_CACHE=<file> keeps the choices across processes (read at the first
// lookup, each new choice appended; a file written by another library
// version is started afresh). Keys name the device model, not its index.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "dd_tune.cuh"

namespace dd {
namespace {
std::mutex g_mu;
std::map<std::string, int> g_cache;
bool g_file_loaded = false;
const char *const CACHE_HEADER = "# dd-gb300 tune cache 1 (" __DATE__ ")";

// model name of the current device, spaces replaced (cached per device index)
std::string device_model() {
  static std::mutex mu;
  static std::map<int, std::string> names;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(dev);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop;
  std::string n = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "device";
  for (char &c : n)
    if (c == ' ' || c == '|') c = '_';
  n += "_" + std::to_string(prop.multiProcessorCount);
  names[dev] = n;
  return n;
}

// with g_mu held: read DD_TUNE_CACHE once
void load_file_locked() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char *path = getenv("DD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[512];
  bool ok = fgets(line, sizeof line, f) && strncmp(line, CACHE_HEADER, strlen(CACHE_HEADER)) == 0;
  while (ok && fgets(line, sizeof line, f)) {
    char key[448];
    int v = 0;
    if (sscanf(line, "%447s %d", key, &v) == 2 && v >= 0) g_cache[key] = v;
  }
  fclose(f);
  if (!ok) {   // another version's file: start it afresh
    FILE *w = fopen(path, "w");
    if (w) {
      fprintf(w, "%s\n", CACHE_HEADER);
      fclose(w);
    }
  }
}

// with g_mu held: append one choice to DD_TUNE_CACHE
void append_file_locked(const std::string &key, int v) {
  const char *path = getenv("DD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "a+");
  if (!f) return;
  fseek(f, 0, SEEK_END);
  if (ftell(f) == 0) fprintf(f, "%s\n", CACHE_HEADER);
  fprintf(f, "%s %d\n", key.c_str(), v);
  fclose(f);
}
}  // namespace

std::string tune_key(const char *kind, const Geom &g, int prec, int nrhs) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%s|%d,%d,%d,%d|%d,%d,%d,%d|%d|%d", kind, device_model().c_str(), g.L[0], g.L[1],
           g.L[2], g.L[3], g.bd[0], g.bd[1], g.bd[2], g.bd[3], prec, nrhs);
  return buf;
}

namespace {
thread_local bool t_direct = false;
}
bool direct_launch() { return t_direct; }
DirectLaunch::DirectLaunch() : prev(t_direct) { t_direct = true; }
DirectLaunch::~DirectLaunch() { t_direct = prev; }

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
    load_file_locked();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *chosen = it->second < nvariants ? it->second : 0;
      return DD_OK;
    }
  }
  if (t_direct) {   // no trial launches: the default variant, not cached
    *chosen = 0;
    return DD_OK;
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
  append_file_locked(key, best_v);
  *chosen = best_v;
  return DD_OK;
}

int tune_lookup(const std::string &key) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_file_locked();
  auto it = g_cache.find(key);
  return it == g_cache.end() ? -1 : it->second;
}

}  // namespace dd
