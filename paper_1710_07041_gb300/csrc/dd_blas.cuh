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
  // return the scratch to the workspace cache (no queued work may use it)
  void release_to_pool();
  // h[i] = <V_i, w> (i < k, complex, FP64), *wnorm2 = <w, w>; V_i = V + i * ldv complex
  int mdot(const double *V, size_t ldv, int k, const double *w, size_t n, double *h_dev, double *wnorm2_dev,
           cudaStream_t st);
  // w -= sum_i h_i V_i, *norm2 = <w, w>
  int maxpy_norm(const double *V, size_t ldv, int k, const double *h_dev, double *w, size_t n, double *norm2_dev,
                 cudaStream_t st);
  int norm2(const double *w, size_t n, double *norm2_dev, cudaStream_t st);
  int scale(double *y, const double *x, double a, size_t n, cudaStream_t st);
  int xmy(const double *x, double *y, size_t n, cudaStream_t st);  // y = x - y
  // Double-float (DF) variants: vectors of n complex entries stored as float4
  // (re_hi, im_hi, re_lo, im_lo); V_i = V + i * ldv complex entries.
  // w32 != nullptr: w is the FP32 spinor field w32 (block-major, lvb = log2 of
  // the block volume), read as double-float {value, 0}; df_maxpy_norm then
  // writes the updated vector to w.
  int df_mdot(const float *V, size_t ldv, int k, const float *w, size_t n, double *h_dev, double *wnorm2_dev,
              cudaStream_t st, const float *w32 = nullptr, int lvb = 0);
  // scl (device, optional): the coefficients h_i are multiplied by scl[i]
  // before the update (for a basis stored as v_i = s_i V_i with h_i = <V_i, w>
  // the caller passes s_i^2)
  int df_maxpy_norm(const float *V, size_t ldv, int k, const double *h_dev, float *w, size_t n, double *norm2_dev,
                    cudaStream_t st, const float *w32 = nullptr, int lvb = 0, const double *scl = nullptr);
  int set_double(double *dev, double v, cudaStream_t st);   // *dev = v, stream-ordered
  int df_scale(float *y, const float *x, double a, size_t n, cudaStream_t st);
  int f64_to_df(float *y, const double *x, double a, size_t n, cudaStream_t st);  // y = a x
  // site-wise: DF field -> storage `prec` (scaled), and FP32 field -> DF field
  int df_to_field(const Geom &g, const float *in, int prec, void *out, double scale, cudaStream_t st);
  int field_to_df(const Geom &g, int prec, const void *in, float *out, cudaStream_t st);
  // x += sum_i y_i Z_i, Z fields of precision zprec with zbytes stride
  int update_x(const Geom &g, double *x, int zprec, const void *Z, size_t zbytes, int k, const double *y_dev,
               cudaStream_t st);
};

}  // namespace dd
