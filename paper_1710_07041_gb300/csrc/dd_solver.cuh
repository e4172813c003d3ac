// Outer FGMRES solver internals (see dd_solver.cu).
#pragma once
#include "dd_blas.cuh"

namespace dd {

// Device workspace of one FGMRES(m) solve on one lattice.
struct SolveWork {
  int prec = -1, zprec = -1, m = 0;
  long long V = 0;
  size_t zbytes = 0, pbytes = 0, bytes = 0;
  double *Vb = nullptr;            // (m+1) FP64 basis fields
  void *Z = nullptr;               // m preconditioned fields (zprec)
  double *w = nullptr, *r = nullptr, *x = nullptr, *b = nullptr, *tmp = nullptr, *canon = nullptr;
  void *tin = nullptr, *tout = nullptr, *zt = nullptr;
  double *hdev = nullptr, *ydev = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  Blas blas;
  ~SolveWork();
  void release();
  int ensure(const Geom &g, int prec, int m);
  static size_t bytes_needed(const Geom &g, int prec, int m);
};

int check_solve_params(const dd_solve_params *p);
int fgmres_one(const Op *op, const dd_solve_params &p, SolveWork &W, dd_solve_info &info, cudaStream_t st,
               const volatile int *cancel);
int solve_canonical(const Op *op, const dd_solve_params &p, const double *b, double *x, int nrhs,
                    dd_solve_info *info, cudaStream_t st, SolveWork &W, const volatile int *cancel);

}  // namespace dd
