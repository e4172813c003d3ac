// Two-level aggregation multigrid internals (see dd_mg.cu).
#pragma once
#include <map>
#include <string>
#include <utility>

#include "dd_blas.cuh"

namespace dd {

constexpr int MAGIC_MG = 0x4d475231;
struct Mg;

// Device workspace of one stream's two-level preconditioner applications.
struct MgWork {
  size_t nc = 0;               // coarse vector length (complex)
  float2 *Vc = nullptr;        // coarse Krylov basis (kmax + 1 vectors)
  float2 *w = nullptr, *w2 = nullptr, *cb = nullptr, *ce = nullptr;
  float *xf = nullptr, *rf = nullptr, *tf = nullptr;   // fine FP32 fields
  void *tin = nullptr, *tout = nullptr;                // smoother-precision fields
  float2 *partial = nullptr;   // coarse reduction partials
  float *pnorm = nullptr;
  void *st = nullptr;          // coarse GMRES control state (device)
  bool warm = false;           // one eager application done (variants tuned)
  std::map<std::string, std::pair<cudaGraphExec_t, size_t>> graphs;   // (r, x, scale) -> graph, nodes
  ~MgWork();
  int init(const Mg *mg);
  static size_t bytes(const Geom &g, int prec, int N, int kmax);
};

struct Mg {
  int magic;
  Op *op;
  dd_mg_params p;
  int N;                 // test vectors
  float *V = nullptr;    // N FP32 fields: orthonormal per (aggregate, chirality); set-up only
  __half *Vh = nullptr;  // the same N fields rounded to FP16: the interpolation P
  __half2 *Dc = nullptr; // coarse operator [aggregate][9][col][row padded to 4], complex FP16
  MgWork work;           // for the dd_mg_* entry points
};

int mg_restrict(const Mg *mg, const float *in, float2 *out, cudaStream_t st);
int mg_prolong(const Mg *mg, const float2 *c, float *out, cudaStream_t st);
int mg_coarse_apply(const Mg *mg, const float2 *x, float2 *y, cudaStream_t st);
int mg_coarse_solve(const Mg *mg, MgWork &W, const float2 *b, float2 *e, cudaStream_t st);
// x = scale * M r for FP32 fields r, x
int mg_apply(const Mg *mg, MgWork &W, const float *r, float *x, cudaStream_t st, float scale = 1.0f);
void destroy_mg(void *h);

}  // namespace dd
