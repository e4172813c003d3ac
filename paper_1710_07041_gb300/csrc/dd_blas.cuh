// FP64 vector operations of the outer solver (see dd_blas.cu).
#pragma once
#include "dd_internal.cuh"

namespace dd {

// Owns the scratch of the two-stage reductions for one stream of work.
struct Blas {
  int nblk = 0;
  double *partial = nullptr;  // [nblk][33] per-block partial sums
  double *result = nullptr;   // [256] reduced values
  double *hpin = nullptr;     // pinned host mirror
  ~Blas();
  int init(int sms);
  // h[i] = <V_i, w> (i < k, complex, FP64), *wnorm2 = <w, w>; V_i = V + i * ldv complex
  int mdot(const double *V, size_t ldv, int k, const double *w, size_t n, double *h_dev, double *wnorm2_dev,
           cudaStream_t st);
  // w -= sum_i h_i V_i, *norm2 = <w, w>
  int maxpy_norm(const double *V, size_t ldv, int k, const double *h_dev, double *w, size_t n, double *norm2_dev,
                 cudaStream_t st);
  int norm2(const double *w, size_t n, double *norm2_dev, cudaStream_t st);
  int scale(double *y, const double *x, double a, size_t n, cudaStream_t st);
  int xmy(const double *x, double *y, size_t n, cudaStream_t st);  // y = x - y
  // x += sum_i y_i Z_i, Z fields of precision zprec with zbytes stride
  int update_x(const Geom &g, double *x, int zprec, const void *Z, size_t zbytes, int k, const double *y_dev,
               cudaStream_t st);
};

}  // namespace dd
