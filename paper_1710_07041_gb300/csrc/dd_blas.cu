// FP64 vector kernels of the outer FGMRES (Arnoldi orthogonalisation, norms,
// solution update). Vectors are FP64 fields viewed as flat arrays of complex
// numbers (all FP64 fields share one element order). Reductions are two-stage
// with a fixed grid and a fixed summation order, so every result is
// bit-reproducible and independent of what else runs on the device.
#include "dd_blas.cuh"

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

// out[i] = sum_b partial[b][i], i < nv, fixed order
__global__ void k_sum_partials(const double *partial, int nblk, int stride, int nv, double *out) {
  int i = threadIdx.x;
  if (i >= nv) return;
  double s = 0;
  for (int b = 0; b < nblk; b++) s += partial[(size_t)b * stride + i];
  out[i] = s;
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

}  // namespace

Blas::~Blas() {
  if (partial) cudaFree(partial);
  if (result) cudaFree(result);
  if (hpin) cudaFreeHost(hpin);
}

int Blas::init(int sms) {
  nblk = sms > 0 ? 4 * sms : 608;
  DD_CUDA(cudaMalloc(&partial, sizeof(double) * (size_t)nblk * (2 * 16 + 1)));
  DD_CUDA(cudaMalloc(&result, sizeof(double) * 256));
  DD_CUDA(cudaMallocHost(&hpin, sizeof(double) * 256));
  return DD_OK;
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
    k_sum_partials<<<1, 64, 0, st>>>(partial, nblk, stride, stride, result);
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
  k_sum_partials<<<1, 32, 0, st>>>(partial, nblk, 1, 1, norm2_dev);
  DD_LAUNCHED();
  return DD_OK;
}

int Blas::norm2(const double *w, size_t n, double *norm2_dev, cudaStream_t st) {
  k_mdot<4><<<nblk, RED_TPB, 0, st>>>((const double2 *)w, 0, 0, (const double2 *)w, n, partial);
  DD_LAUNCHED();
  k_sum_partials<<<1, 32, 0, st>>>(partial, nblk, 9, 9, result);
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

int Blas::update_x(const Geom &g, double *x, int zprec, const void *Z, size_t zbytes, int k, const double *y_dev,
                   cudaStream_t st) {
  unsigned grid = (unsigned)((g.V + 127) / 128);
  switch (zprec) {
    case DD_F64: k_update_x<double><<<grid, 128, 0, st>>>(g, x, Z, zbytes, k, (const double2 *)y_dev); break;
    case DD_F32: k_update_x<float><<<grid, 128, 0, st>>>(g, x, Z, zbytes, k, (const double2 *)y_dev); break;
    default: set_error("update_x: bad precision"); return DD_EINVAL;
  }
  return launched("k_update_x");
}

}  // namespace dd
