// Launch-configuration autotuner (see dd_tune.cu).
#pragma once
#include <functional>
#include <string>

#include "dd_internal.cuh"

namespace dd {
std::string tune_key(const char *kind, const Geom &g, int prec, int nrhs);
// Pick (and cache under `key`) the fastest of `nvariants` launch variants;
// run(v) enqueues variant v on stream st. *chosen receives the choice.
int tuned_variant(const std::string &key, int nvariants, const std::function<int(int)> &run, cudaStream_t st,
                  int *chosen);
int tune_lookup(const std::string &key);  // cached choice or -1

// Launches without set-up work, for calls that promise to allocate nothing
// (dd_solve_noalloc). While a DirectLaunch object lives on a thread, that
// thread's launch-variant choices come from the tuner's cache only (variant 0
// on a miss, which is not cached, so later ordinary calls still tune) and the
// Schwarz smoother's launches are enqueued directly instead of through a
// cached CUDA graph (no capture, no instantiation).
bool direct_launch();
struct DirectLaunch {
  DirectLaunch();
  ~DirectLaunch();
  DirectLaunch(const DirectLaunch &) = delete;
  DirectLaunch &operator=(const DirectLaunch &) = delete;
  bool prev;
};
}  // namespace dd
