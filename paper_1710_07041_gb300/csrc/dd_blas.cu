// FP64 vector kernels of the outer FGMRES (Arnoldi orthogonalisation, norms,
// solution update). Vectors are FP64 fields viewed as flat arrays of complex
// numbers (all FP64 fields share one element order). Reductions are two-stage
// with a fixed grid and a fixed summation order, so every result is
// bit-reproducible and independent of what else runs on the device.
#include "dd_blas.cuh"
#include "dd_pool.cuh"

namespace dd {
namespace {

constexpr int RED_TPB = 256;

__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
  // acc += conj(a) * b
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
  return acc;
}

// Block-reduce NV doubles held per thread into red[NV] (fixed order).
template <int NV>
__device__ __forceinline__ void block_reduce(double *v, double *smem, double *out) {
#pragma unroll
  for (int i = 0; i < NV; i++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < NV; i++) smem[i * 32 + w] = v[i];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0;
    for (int k = 0; k < nw; k++) s += smem[threadIdx.x * 32 + k];
    out[threadIdx.x] = s;
  }
}

// partial[blk][0..2k+1] = this block's sums of conj(V_i) w (i < k) and |w|^2
template <int KMAX>
__global__ void __launch_bounds__(RED_TPB) k_mdot(const double2 *__restrict__ V, size_t ldv, int k,
                                                  const double2 *__restrict__ w, size_t n, double *partial) {
  __shared__ double smem[(2 * KMAX + 1) * 32];
  double acc[2 * KMAX + 1];
#pragma unroll
  for (int i = 0; i < 2 * KMAX + 1; i++) acc[i] = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 we = w[e];
    acc[2 * KMAX] = fma(we.x, we.x, fma(we.y, we.y, acc[2 * KMAX]));
#pragma unroll
    for (int i = 0; i < KMAX; i++) {
      if (i < k) {
        double2 a = cfma_conj(V[i * ldv + e], we, make_double2(acc[2 * i], acc[2 * i + 1]));
        acc[2 * i] = a.x;
        acc[2 * i + 1] = a.y;
      }
    }
  }
  block_reduce<2 * KMAX + 1>(acc, smem, partial + (size_t)blockIdx.x * (2 * KMAX + 1));
}

// w -= sum_i h_i V_i (h complex, device); partial[blk] = block's |w|^2
template <int KMAX>
__global__ void __launch_bounds__(RED_TPB) k_maxpy_norm(const double2 *__restrict__ V, size_t ldv, int k,
                                                        const double2 *__restrict__ h, double2 *w, size_t n,
                                                        double *partial) {
  __shared__ double smem[32];
  __shared__ double2 hs[KMAX];
  if (threadIdx.x < KMAX) hs[threadIdx.x] = threadIdx.x < k ? h[threadIdx.x] : make_double2(0, 0);
  __syncthreads();
  double acc[1] = {0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 we = w[e];
#pragma unroll
    for (int i = 0; i < KMAX; i++) {
      if (i < k) {
        double2 v = V[i * ldv + e], c = hs[i];
        we.x -= c.x * v.x - c.y * v.y;
        we.y -= c.x * v.y + c.y * v.x;
      }
    }
    w[e] = we;
    acc[0] = fma(we.x, we.x, fma(we.y, we.y, acc[0]));
  }
  block_reduce<1>(acc, smem, partial + blockIdx.x);
}

// out[i] = sum_b partial[b][i]: one CTA per value i, fixed summation order
// (thread t sums blocks t, t + 256, ..., then a fixed-shape tree)
__global__ void __launch_bounds__(256) k_sum_partials(const double *partial, int nblk, int stride, int nv,
                                                      double *out) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  if (i >= nv) return;
  double s = 0;
  for (int b = threadIdx.x; b < nblk; b += 256) s += partial[(size_t)b * stride + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}

__global__ void k_scale(double2 *y, const double2 *x, double a, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 v = x[e];
    y[e] = make_double2(a * v.x, a * v.y);
  }
}

// y = x - y
__global__ void k_xmy(const double2 *x, double2 *y, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 a = x[e], b = y[e];
    y[e] = make_double2(a.x - b.x, a.y - b.y);
  }
}

// x(site) += sum_i y_i Z_i(site), Z in storage SZ (its own layout), x FP64
template <typename SZ>
__global__ void k_update_x(Geom g, double *x, const void *Z, size_t zbytes, int k, const double2 *__restrict__ y) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  using C = typename Store<SZ>::comp_t;
  Spinor<double> acc;
  load_spinor<double, double>(x, g, b, s, acc);
  for (int i = 0; i < k; i++) {
    Spinor<C> z;
    load_spinor<SZ, C>((const char *)Z + i * zbytes, g, b, s, z);
    double2 c = y[i];
#pragma unroll
    for (int q = 0; q < 12; q++) {
      double zr = (double)z.c[q].re, zi = (double)z.c[q].im;
      acc.c[q].re += c.x * zr - c.y * zi;
      acc.c[q].im += c.x * zi + c.y * zr;
    }
  }
  store_spinor<double, double>(x, g, b, s, acc);
}


// ------------------------------------------------------------------------
// Double-float ("DF") vectors: each complex entry is a float4
// (re_hi, im_hi, re_lo, im_lo) whose value is hi + lo, a 48-bit significand.
// GB300 executes FP64 at a small fraction of its FP32 rate, so FP64 dot
// products over the Krylov basis are ALU-bound; DF arithmetic built from
// error-free FP32 transformations (Dekker's product, Knuth's TwoSum) keeps
// FP64-class accuracy at FP32 throughput, so these kernels stay HBM-bound.

struct df { float h, l; };

// s += a * b   (a, b double-float; lazy accumulation: error terms collected in s.l)
__device__ __forceinline__ void df_mac(df &s, float ah, float al, float bh, float bl) {
  float p = ah * bh;
  float pe = fmaf(ah, bh, -p);                  // exact error of the product
  float c = fmaf(ah, bl, al * bh);              // cross terms
  float t = s.h + p;                            // TwoSum(s.h, p)
  float z = t - s.h;
  float e = (s.h - (t - z)) + (p - z);
  s.h = t;
  s.l += e + pe + c;
}
// s -= a * b
__device__ __forceinline__ void df_msub(df &s, float ah, float al, float bh, float bl) {
  df_mac(s, -ah, -al, bh, bl);
}
__device__ __forceinline__ double df_val(const df &s) { return (double)s.h + (double)s.l; }
__device__ __forceinline__ df df_norm(float h, float l) {
  float t = h + l;
  return {t, l - (t - h)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  float t = a.h + b.h;
  float z = t - a.h;
  float e = (a.h - (t - z)) + (b.h - z);
  return {t, a.l + b.l + e};
}

// Block-reduce NV double-float values: warp shuffles in DF, then the warp
// leaders' results in FP64 (fixed order).
template <int NV>
__device__ __forceinline__ void block_reduce_df(df *v, double *smem, double *out) {
#pragma unroll
  for (int i = 0; i < NV; i++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df u = {__shfl_xor_sync(0xffffffffu, v[i].h, o), __shfl_xor_sync(0xffffffffu, v[i].l, o)};
      v[i] = df_add(v[i], u);
    }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < NV; i++) smem[i * 32 + w] = df_val(v[i]);
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0;
    for (int k = 0; k < nw; k++) s += smem[threadIdx.x * 32 + k];
    out[threadIdx.x] = s;
  }
}

// Element e of a DF vector (complex number c of site s in block b, at
// e = (b * 12 + c) * Vb + s) read from an FP32 spinor field instead, as the
// double-float {value, 0}: the Arnoldi vector w = D z straight from the FP32
// Dslash, without a conversion pass (lvb = log2 Vb).
__device__ __forceinline__ float4 w_from_f32(const float *w32, size_t e, int lvb) {
  const size_t s = e & (((size_t)1 << lvb) - 1), q = e >> lvb;
  const size_t c = q % 12, b = q / 12;
  const float2 v = *(const float2 *)(w32 + ((((b * 6 + (c >> 1)) << lvb) + s) << 2) + ((c & 1) << 1));
  return make_float4(v.x, v.y, 0.f, 0.f);
}
template <bool W32>
__device__ __forceinline__ float4 w_at(const float4 *w, const float *w32, size_t e, int lvb) {
  if constexpr (W32) return w_from_f32(w32, e, lvb);
  return w[e];
}

// partial[blk] = this block's sums of conj(V_i) w (i < k) and |w|^2, as doubles.
// Two elements per thread and iteration keep more loads in flight. W32: w is
// read from the FP32 field w32 (see w_from_f32).
template <int KMAX, bool W32 = false>
__global__ void __launch_bounds__(RED_TPB) k_df_mdot(const float4 *__restrict__ V, size_t ldv, int k,
                                                     const float4 *__restrict__ w, size_t n, double *partial,
                                                     const float *__restrict__ w32 = nullptr, int lvb = 0) {
  __shared__ double smem[(2 * KMAX + 1) * 32];
  df acc[2 * KMAX + 1];
#pragma unroll
  for (int i = 0; i < 2 * KMAX + 1; i++) acc[i] = {0.f, 0.f};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += 2 * stride) {
    const size_t e2 = e + stride;
    const bool two = e2 < n;
    float4 we = w_at<W32>(w, w32, e, lvb), we2 = two ? w_at<W32>(w, w32, e2, lvb) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v[KMAX], v2[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; i++)
      if (i < k) {
        v[i] = V[i * ldv + e];
        v2[i] = two ? V[i * ldv + e2] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    df_mac(acc[2 * KMAX], we.x, we.z, we.x, we.z);
    df_mac(acc[2 * KMAX], we.y, we.w, we.y, we.w);
    df_mac(acc[2 * KMAX], we2.x, we2.z, we2.x, we2.z);
    df_mac(acc[2 * KMAX], we2.y, we2.w, we2.y, we2.w);
#pragma unroll
    for (int i = 0; i < KMAX; i++) {
      if (i < k) {
        // re += vr wr + vi wi ; im += vr wi - vi wr
        df_mac(acc[2 * i], v[i].x, v[i].z, we.x, we.z);
        df_mac(acc[2 * i], v[i].y, v[i].w, we.y, we.w);
        df_mac(acc[2 * i + 1], v[i].x, v[i].z, we.y, we.w);
        df_msub(acc[2 * i + 1], v[i].y, v[i].w, we.x, we.z);
        df_mac(acc[2 * i], v2[i].x, v2[i].z, we2.x, we2.z);
        df_mac(acc[2 * i], v2[i].y, v2[i].w, we2.y, we2.w);
        df_mac(acc[2 * i + 1], v2[i].x, v2[i].z, we2.y, we2.w);
        df_msub(acc[2 * i + 1], v2[i].y, v2[i].w, we2.x, we2.z);
      }
    }
  }
  block_reduce_df<2 * KMAX + 1>(acc, smem, partial + (size_t)blockIdx.x * (2 * KMAX + 1));
}

// w -= sum_i h_i V_i (h complex doubles on the device); partial[blk] = |w|^2.
// W32: the input w is read from the FP32 field w32 (see w_from_f32) and the
// result written to w.
template <int KMAX, bool W32 = false>
__global__ void __launch_bounds__(RED_TPB) k_df_maxpy_norm(const float4 *__restrict__ V, size_t ldv, int k,
                                                           const double2 *__restrict__ h, float4 *w, size_t n,
                                                           double *partial, const float *__restrict__ w32 = nullptr,
                                                           int lvb = 0, const double *__restrict__ scl = nullptr) {
  __shared__ double smem[32];
  __shared__ float4 hs[KMAX];   // (re_hi, im_hi, re_lo, im_lo)
  if (threadIdx.x < KMAX) {
    double2 c = threadIdx.x < k ? h[threadIdx.x] : make_double2(0, 0);
    if (scl && threadIdx.x < k) {   // per-vector coefficient factor (see Blas::df_maxpy_norm)
      c.x *= scl[threadIdx.x];
      c.y *= scl[threadIdx.x];
    }
    float rh = (float)c.x, ih = (float)c.y;
    hs[threadIdx.x] = make_float4(rh, ih, (float)(c.x - rh), (float)(c.y - ih));
  }
  __syncthreads();
  df nrm = {0.f, 0.f};
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += 2 * stride) {
    const size_t e2 = e + stride;
    const bool two = e2 < n;
    float4 we = w_at<W32>(w, w32, e, lvb), we2 = two ? w_at<W32>(w, w32, e2, lvb) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v[KMAX], v2[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; i++)
      if (i < k) {
        v[i] = V[i * ldv + e];
        v2[i] = two ? V[i * ldv + e2] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    df re = {we.x, we.z}, im = {we.y, we.w}, re2 = {we2.x, we2.z}, im2 = {we2.y, we2.w};
#pragma unroll
    for (int i = 0; i < KMAX; i++) {
      if (i < k) {
        const float4 c = hs[i];
        // w -= c v : re -= cr vr - ci vi ; im -= cr vi + ci vr
        df_msub(re, c.x, c.z, v[i].x, v[i].z);
        df_mac(re, c.y, c.w, v[i].y, v[i].w);
        df_msub(im, c.x, c.z, v[i].y, v[i].w);
        df_msub(im, c.y, c.w, v[i].x, v[i].z);
        df_msub(re2, c.x, c.z, v2[i].x, v2[i].z);
        df_mac(re2, c.y, c.w, v2[i].y, v2[i].w);
        df_msub(im2, c.x, c.z, v2[i].y, v2[i].w);
        df_msub(im2, c.y, c.w, v2[i].x, v2[i].z);
      }
    }
    re = df_norm(re.h, re.l);
    im = df_norm(im.h, im.l);
    w[e] = make_float4(re.h, im.h, re.l, im.l);
    df_mac(nrm, re.h, re.l, re.h, re.l);
    df_mac(nrm, im.h, im.l, im.h, im.l);
    if (two) {
      re2 = df_norm(re2.h, re2.l);
      im2 = df_norm(im2.h, im2.l);
      w[e2] = make_float4(re2.h, im2.h, re2.l, im2.l);
      df_mac(nrm, re2.h, re2.l, re2.h, re2.l);
      df_mac(nrm, im2.h, im2.l, im2.h, im2.l);
    }
  }
  block_reduce_df<1>(&nrm, smem, partial + blockIdx.x);
}

// y = a x (DF), a double
__global__ void k_df_scale(float4 *y, const float4 *x, double a, size_t n) {
  const float ah = (float)a, al = (float)(a - (double)ah);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float4 v = x[e];
    df re = {0.f, 0.f}, im = {0.f, 0.f};
    df_mac(re, ah, al, v.x, v.z);
    df_mac(im, ah, al, v.y, v.w);
    re = df_norm(re.h, re.l);
    im = df_norm(im.h, im.l);
    y[e] = make_float4(re.h, im.h, re.l, im.l);
  }
}

// y (DF) = a x (FP64)
__global__ void k_f64_to_df(float4 *y, const double2 *x, double a, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double2 v = x[e];
    double r = a * v.x, i = a * v.y;
    float rh = (float)r, ih = (float)i;
    y[e] = make_float4(rh, ih, (float)(r - rh), (float)(i - ih));
  }
}

// Site-wise conversions between a DF field (FP64 chunk positions) and a
// field of storage S: out = scale * in.
template <typename S>
__global__ void k_df_to_field(Geom g, const float4 *__restrict__ in, void *out, float scale) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  Spinor<float> v;
#pragma unroll
  for (int c = 0; c < 12; c++) {
    float4 q = in[((size_t)b * 12 + c) * g.Vb + s];
    v.c[c] = {(q.x + q.z) * scale, (q.y + q.w) * scale};
  }
  store_spinor<S, float>(out, g, b, s, v);
}

template <typename S>
__global__ void k_field_to_df(Geom g, const void *in, float4 *__restrict__ out) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  Spinor<float> v;
  load_spinor<S, float>(in, g, b, s, v);
#pragma unroll
  for (int c = 0; c < 12; c++) out[((size_t)b * 12 + c) * g.Vb + s] = make_float4(v.c[c].re, v.c[c].im, 0.f, 0.f);
}

// x(site) += sum_i y_i Z_i(site) for FP32 Z: the sum is accumulated in
// double-float (y_i split into hi/lo floats once per CTA), then added to the
// FP64 x with one FP64 add per real.
__global__ void __launch_bounds__(128) k_update_x_df(Geom g, double *x, const void *Z, size_t zbytes, int k,
                                                     const double2 *__restrict__ y) {
  __shared__ float4 ys[64];
  if (threadIdx.x < 64 && (int)threadIdx.x < k) {
    double2 c = y[threadIdx.x];
    float rh = (float)c.x, ih = (float)c.y;
    ys[threadIdx.x] = make_float4(rh, ih, (float)(c.x - rh), (float)(c.y - ih));
  }
  __syncthreads();
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  df re[12], im[12];
#pragma unroll
  for (int q = 0; q < 12; q++) re[q] = im[q] = {0.f, 0.f};
  for (int i = 0; i < k; i++) {
    Spinor<float> z;
    load_spinor<float, float>((const char *)Z + i * zbytes, g, b, s, z);
    const float4 c = ys[i];
#pragma unroll
    for (int q = 0; q < 12; q++) {
      // (cr + i ci)(zr + i zi)
      df_mac(re[q], c.x, c.z, z.c[q].re, 0.f);
      df_msub(re[q], c.y, c.w, z.c[q].im, 0.f);
      df_mac(im[q], c.x, c.z, z.c[q].im, 0.f);
      df_mac(im[q], c.y, c.w, z.c[q].re, 0.f);
    }
  }
  Spinor<double> acc;
  load_spinor<double, double>(x, g, b, s, acc);
#pragma unroll
  for (int q = 0; q < 12; q++) {
    acc.c[q].re += df_val(re[q]);
    acc.c[q].im += df_val(im[q]);
  }
  store_spinor<double, double>(x, g, b, s, acc);
}

}  // namespace

Blas::~Blas() {
  if (partial) cudaFree(partial);
  if (result) cudaFree(result);
  if (hpin) cudaFreeHost(hpin);
}

int Blas::init(int sms) {
  nblk = sms > 0 ? 4 * sms : 608;
  partial = (double *)pool_dev_alloc(sizeof(double) * (size_t)nblk * (2 * 16 + 1));
  result = (double *)pool_dev_alloc(sizeof(double) * 256);
  hpin = (double *)pool_host_alloc(sizeof(double) * 256);
  if (!partial || !result || !hpin) {
    set_error("blas: out of memory for reduction scratch");
    return DD_ENOMEM;
  }
  return DD_OK;
}

void Blas::release_to_pool() {
  pool_dev_free(partial, sizeof(double) * (size_t)nblk * (2 * 16 + 1));
  pool_dev_free(result, sizeof(double) * 256);
  pool_host_free(hpin, sizeof(double) * 256);
  partial = result = hpin = nullptr;
}

int Blas::mdot(const double *V, size_t ldv, int k, const double *w, size_t n, double *h_dev, double *wnorm2_dev,
               cudaStream_t st) {
  // in groups of up to 16 vectors
  for (int i0 = 0; i0 < k || (k == 0 && i0 == 0); i0 += 16) {
    int kk = k - i0 < 16 ? k - i0 : 16;
    if (kk < 0) kk = 0;
    const double2 *Vi = (const double2 *)V + (size_t)i0 * ldv;
    if (kk <= 4)
      k_mdot<4><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, (const double2 *)w, n, partial);
    else
      k_mdot<16><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, (const double2 *)w, n, partial);
    int stride = kk <= 4 ? 9 : 33;
    DD_LAUNCHED();
    k_sum_partials<<<stride, 256, 0, st>>>(partial, nblk, stride, stride, result);
    DD_LAUNCHED();
    if (kk > 0) DD_CUDA(cudaMemcpyAsync(h_dev + 2 * i0, result, sizeof(double) * 2 * kk, cudaMemcpyDeviceToDevice, st));
    if (wnorm2_dev && i0 == 0)
      DD_CUDA(cudaMemcpyAsync(wnorm2_dev, result + (stride - 1), sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (k == 0) break;
  }
  return DD_OK;
}

int Blas::maxpy_norm(const double *V, size_t ldv, int k, const double *h_dev, double *w, size_t n, double *norm2_dev,
                     cudaStream_t st) {
  for (int i0 = 0; i0 < k; i0 += 16) {
    int kk = k - i0 < 16 ? k - i0 : 16;
    const double2 *Vi = (const double2 *)V + (size_t)i0 * ldv;
    const double2 *hi = (const double2 *)h_dev + i0;
    if (kk <= 4)
      k_maxpy_norm<4><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, hi, (double2 *)w, n, partial);
    else
      k_maxpy_norm<16><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, hi, (double2 *)w, n, partial);
    DD_LAUNCHED();
  }
  if (k == 0) return norm2(w, n, norm2_dev, st);
  k_sum_partials<<<1, 256, 0, st>>>(partial, nblk, 1, 1, norm2_dev);
  DD_LAUNCHED();
  return DD_OK;
}

int Blas::norm2(const double *w, size_t n, double *norm2_dev, cudaStream_t st) {
  k_mdot<4><<<nblk, RED_TPB, 0, st>>>((const double2 *)w, 0, 0, (const double2 *)w, n, partial);
  DD_LAUNCHED();
  k_sum_partials<<<9, 256, 0, st>>>(partial, nblk, 9, 9, result);
  DD_LAUNCHED();
  DD_CUDA(cudaMemcpyAsync(norm2_dev, result + 8, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return DD_OK;
}

int Blas::scale(double *y, const double *x, double a, size_t n, cudaStream_t st) {
  k_scale<<<nblk, RED_TPB, 0, st>>>((double2 *)y, (const double2 *)x, a, n);
  return launched("k_scale");
}

int Blas::xmy(const double *x, double *y, size_t n, cudaStream_t st) {
  k_xmy<<<nblk, RED_TPB, 0, st>>>((const double2 *)x, (double2 *)y, n);
  return launched("k_xmy");
}

int Blas::df_mdot(const float *V, size_t ldv, int k, const float *w, size_t n, double *h_dev, double *wnorm2_dev,
                  cudaStream_t st, const float *w32, int lvb) {
  for (int i0 = 0; i0 < k || (k == 0 && i0 == 0); i0 += 8) {
    int kk = k - i0 < 8 ? k - i0 : 8;
    if (kk < 0) kk = 0;
    const float4 *Vi = (const float4 *)V + (size_t)i0 * ldv;
    if (w32) {
      if (kk <= 4)
        k_df_mdot<4, true><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, nullptr, n, partial, w32, lvb);
      else
        k_df_mdot<8, true><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, nullptr, n, partial, w32, lvb);
    } else if (kk <= 4)
      k_df_mdot<4><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, (const float4 *)w, n, partial);
    else
      k_df_mdot<8><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, (const float4 *)w, n, partial);
    int stride = kk <= 4 ? 9 : 17;
    DD_LAUNCHED();
    k_sum_partials<<<stride, 256, 0, st>>>(partial, nblk, stride, stride, result);
    DD_LAUNCHED();
    if (kk > 0) DD_CUDA(cudaMemcpyAsync(h_dev + 2 * i0, result, sizeof(double) * 2 * kk, cudaMemcpyDeviceToDevice, st));
    if (wnorm2_dev && i0 == 0)
      DD_CUDA(cudaMemcpyAsync(wnorm2_dev, result + (stride - 1), sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (k == 0) break;
  }
  return DD_OK;
}

int Blas::df_maxpy_norm(const float *V, size_t ldv, int k, const double *h_dev, float *w, size_t n, double *norm2_dev,
                        cudaStream_t st, const float *w32, int lvb, const double *scl) {
  if (k == 0) return df_mdot(V, ldv, 0, w, n, nullptr, norm2_dev, st, w32, lvb);
  for (int i0 = 0; i0 < k; i0 += 8) {
    int kk = k - i0 < 8 ? k - i0 : 8;
    const float4 *Vi = (const float4 *)V + (size_t)i0 * ldv;
    const double2 *hi = (const double2 *)h_dev + i0;
    const double *si = scl ? scl + i0 : nullptr;
    // the first chunk reads the FP32 input (when given) and writes w; later chunks update w
    const bool from32 = w32 && i0 == 0;
    if (from32) {
      if (kk <= 4)
        k_df_maxpy_norm<4, true><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, hi, (float4 *)w, n, partial, w32, lvb, si);
      else
        k_df_maxpy_norm<8, true><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, hi, (float4 *)w, n, partial, w32, lvb, si);
    } else if (kk <= 4)
      k_df_maxpy_norm<4><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, hi, (float4 *)w, n, partial, nullptr, 0, si);
    else
      k_df_maxpy_norm<8><<<nblk, RED_TPB, 0, st>>>(Vi, ldv, kk, hi, (float4 *)w, n, partial, nullptr, 0, si);
    DD_LAUNCHED();
  }
  k_sum_partials<<<1, 256, 0, st>>>(partial, nblk, 1, 1, norm2_dev);
  return launched("k_sum_partials");
}

__global__ void k_set_double(double *p, double v) { *p = v; }
int Blas::set_double(double *dev, double v, cudaStream_t st) {
  k_set_double<<<1, 1, 0, st>>>(dev, v);
  return launched("k_set_double");
}

int Blas::df_scale(float *y, const float *x, double a, size_t n, cudaStream_t st) {
  k_df_scale<<<nblk, RED_TPB, 0, st>>>((float4 *)y, (const float4 *)x, a, n);
  return launched("k_df_scale");
}

int Blas::f64_to_df(float *y, const double *x, double a, size_t n, cudaStream_t st) {
  k_f64_to_df<<<nblk, RED_TPB, 0, st>>>((float4 *)y, (const double2 *)x, a, n);
  return launched("k_f64_to_df");
}

int Blas::df_to_field(const Geom &g, const float *in, int prec, void *out, double scale, cudaStream_t st) {
  unsigned grid = (unsigned)((g.V + 127) / 128);
  const float4 *x = (const float4 *)in;
  switch (prec) {
    case DD_F32: k_df_to_field<float><<<grid, 128, 0, st>>>(g, x, out, (float)scale); break;
    case DD_F16: k_df_to_field<__half><<<grid, 128, 0, st>>>(g, x, out, (float)scale); break;
    case DD_BF16: k_df_to_field<__nv_bfloat16><<<grid, 128, 0, st>>>(g, x, out, (float)scale); break;
    case DD_F16N: k_df_to_field<hn16><<<grid, 128, 0, st>>>(g, x, out, (float)scale); break;
    default: set_error("df_to_field: bad precision"); return DD_EINVAL;
  }
  return launched("k_df_to_field");
}

int Blas::field_to_df(const Geom &g, int prec, const void *in, float *out, cudaStream_t st) {
  unsigned grid = (unsigned)((g.V + 127) / 128);
  switch (prec) {
    case DD_F32: k_field_to_df<float><<<grid, 128, 0, st>>>(g, in, (float4 *)out); break;
    default: set_error("field_to_df: bad precision"); return DD_EINVAL;
  }
  return launched("k_field_to_df");
}

int Blas::update_x(const Geom &g, double *x, int zprec, const void *Z, size_t zbytes, int k, const double *y_dev,
                   cudaStream_t st) {
  unsigned grid = (unsigned)((g.V + 127) / 128);
  switch (zprec) {
    case DD_F64: k_update_x<double><<<grid, 128, 0, st>>>(g, x, Z, zbytes, k, (const double2 *)y_dev); break;
    case DD_F32:
      if (k > 64) {
        set_error("update_x: at most 64 vectors");
        return DD_EINVAL;
      }
      k_update_x_df<<<grid, 128, 0, st>>>(g, x, Z, zbytes, k, (const double2 *)y_dev);
      break;
    default: set_error("update_x: bad precision"); return DD_EINVAL;
  }
  return launched("k_update_x");
}

}  // namespace dd
