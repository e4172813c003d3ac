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
}  // namespace dd
