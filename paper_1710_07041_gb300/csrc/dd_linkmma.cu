// Measurement of the tensor-core question for the multi-right-hand-side link
// product (no counterpart in the paper, whose Schwarz method runs on KNC/KNL
// vector units, Sec. 3.1).
//
// In a Schwarz block with a tile of k right-hand sides, every hop multiplies
// one 3x3 complex link U by 2k complex colour vectors (two spin components
// per right-hand side). In real arithmetic that is the 6x6 matrix
// M = [[Re U, -Im U], [Im U, Re U]] times a 6 x 2k matrix: a contraction of
// length 6. The densest tensor-core form available to a thread block is the
// warp-level mma.sync m16n8k16 (FP16 inputs, FP32 accumulation) with the
// matrices of two site-directions placed block-diagonally in one 16x16 A
// operand (rows and columns 0-5 and 6-11, the rest zero): 2 x 36 of its 256
// entries are useful, and each B operand holds 8 of the 2k columns of both
// sites. (tcgen05 tiles start at M = 64, where the same packing is sparser
// still.) This file times that form against the FP32 CUDA-core form on the
// same products, both with their operands in shared memory, for k = 12.
//
//   method 0: FP32 operands, FP32 arithmetic (thread per site-direction
//             and 6 of its 24 columns);
//   method 1: FP16 operands, mma.sync with the block-diagonal packing, FP32
//             accumulation (warp per pair of site-directions);
//   method 2: FP16 operands converted to FP32 on load, FP32 arithmetic (the
//             arithmetic of the Schwarz kernel's 16-bit storage).
//
// Inputs are multiples of 1/64 in [-1, 1], exact in FP16, so all three
// methods compute the same products and differ only by FP32 rounding.
#include <cmath>
#include <cstdio>
#include <vector>

#include "dd_internal.cuh"

namespace dd {
namespace {

constexpr int LQ = 64;       // site-directions per CTA tile
constexpr int LCOLS = 24;    // columns: 12 right-hand sides x 2 spin components
constexpr int LTPB = 256;

// deterministic input in [-1, 1], a multiple of 1/64
__device__ __forceinline__ float probe_value(unsigned i) {
  unsigned h = i * 2654435761u;
  h ^= h >> 15;
  h *= 2246822519u;
  h ^= h >> 13;
  return (float)((int)(h % 129u) - 64) / 64.f;
}

// Tile of one CTA: U [LQ][9] complex, X [LQ][LCOLS][3] complex, Y [LQ][LCOLS][3].
template <typename T> struct LinkTile {
  T *u, *x;
  float2 *y;
};

template <typename T> __device__ __forceinline__ float2 ld2(const T *p, int i);
template <> __device__ __forceinline__ float2 ld2<float2>(const float2 *p, int i) { return p[i]; }
template <> __device__ __forceinline__ float2 ld2<__half2>(const __half2 *p, int i) { return __half22float2(p[i]); }

template <typename T>
__device__ void fill_tile(LinkTile<T> t, unsigned base) {
  for (int i = threadIdx.x; i < LQ * 9; i += blockDim.x) {
    const float re = probe_value(base + 2 * i), im = probe_value(base + 2 * i + 1);
    if constexpr (sizeof(T) == 8) t.u[i] = make_float2(re, im);
    else t.u[i] = __floats2half2_rn(re, im);
  }
  for (int i = threadIdx.x; i < LQ * LCOLS * 3; i += blockDim.x) {
    const float re = probe_value(base + 100003u + 2 * i), im = probe_value(base + 100004u + 2 * i);
    if constexpr (sizeof(T) == 8) t.x[i] = make_float2(re, im);
    else t.x[i] = __floats2half2_rn(re, im);
  }
}

// methods 0 and 2: thread (q, c) computes 6 columns of site-direction q
template <typename T>
__global__ void __launch_bounds__(LTPB) k_link_alu(int reps, float2 *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  LinkTile<T> t;
  t.u = (T *)smem;
  t.x = t.u + LQ * 9;
  t.y = (float2 *)(t.x + LQ * LCOLS * 3);
  fill_tile(t, blockIdx.x * 7919u);
  __syncthreads();
  const int q = threadIdx.x >> 2, c0 = (threadIdx.x & 3) * 6;
  for (int r = 0; r < reps; r++) {
    float2 u[9];
#pragma unroll
    for (int i = 0; i < 9; i++) u[i] = ld2(t.u, q * 9 + i);
#pragma unroll
    for (int c = c0; c < c0 + 6; c++) {
      float2 x[3];
#pragma unroll
      for (int k = 0; k < 3; k++) x[k] = ld2(t.x, (q * LCOLS + c) * 3 + k);
#pragma unroll
      for (int i = 0; i < 3; i++) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          a.x = fmaf(u[3 * i + k].x, x[k].x, fmaf(-u[3 * i + k].y, x[k].y, a.x));
          a.y = fmaf(u[3 * i + k].x, x[k].y, fmaf(u[3 * i + k].y, x[k].x, a.y));
        }
        t.y[(q * LCOLS + c) * 3 + i] = a;
      }
    }
    __syncthreads();
  }
  if (out)
    for (int i = threadIdx.x; i < LQ * LCOLS * 3; i += blockDim.x) out[(size_t)blockIdx.x * LQ * LCOLS * 3 + i] = t.y[i];
}

// entry (r, c) of the block-diagonal A operand of the pair (q0, q0 + 1)
__device__ __forceinline__ float a_entry(const __half2 *u, int q0, int r, int c) {
  if (r >= 12 || c >= 12 || (r < 6) != (c < 6)) return 0.f;
  const int site = r / 6, rr = r % 6, cc = c % 6;
  const float2 v = __half22float2(u[(q0 + site) * 9 + 3 * (rr % 3) + (cc % 3)]);
  if ((rr < 3) == (cc < 3)) return v.x;
  return rr < 3 ? -v.y : v.y;
}
// entry (k, n) of the B operand (columns 8 g .. 8 g + 7) of the pair
__device__ __forceinline__ float b_entry(const __half2 *x, int q0, int k, int col) {
  if (k >= 12) return 0.f;
  const int site = k / 6, kk = k % 6;
  const float2 v = __half22float2(x[((q0 + site) * LCOLS + col) * 3 + kk % 3]);
  return kk < 3 ? v.x : v.y;
}
__device__ __forceinline__ unsigned pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *(const unsigned *)&h;
}

// method 1: warp per pair of site-directions, three m16n8k16 products per pair
__global__ void __launch_bounds__(LTPB) k_link_mma(int reps, float2 *out) {
  extern __shared__ __align__(16) unsigned char smem[];
  LinkTile<__half2> t;
  t.u = (__half2 *)smem;
  t.x = t.u + LQ * 9;
  t.y = (float2 *)(t.x + LQ * LCOLS * 3);
  fill_tile(t, blockIdx.x * 7919u);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tg = lane & 3;
  float *yf = (float *)t.y;
  for (int r = 0; r < reps; r++) {
    for (int pr = warp; pr < LQ / 2; pr += LTPB / 32) {
      const int q0 = 2 * pr;
      // A fragment: (g, 2tg..), (g+8, 2tg..), (g, 2tg+8..), (g+8, 2tg+8..)
      unsigned a[4];
      a[0] = pack_h2(a_entry(t.u, q0, g, 2 * tg), a_entry(t.u, q0, g, 2 * tg + 1));
      a[1] = pack_h2(a_entry(t.u, q0, g + 8, 2 * tg), a_entry(t.u, q0, g + 8, 2 * tg + 1));
      a[2] = pack_h2(a_entry(t.u, q0, g, 2 * tg + 8), a_entry(t.u, q0, g, 2 * tg + 9));
      a[3] = pack_h2(a_entry(t.u, q0, g + 8, 2 * tg + 8), a_entry(t.u, q0, g + 8, 2 * tg + 9));
#pragma unroll
      for (int cg = 0; cg < LCOLS / 8; cg++) {
        const int col = 8 * cg + g;   // B: (2tg.., g) and (2tg+8.., g)
        unsigned b[2];
        b[0] = pack_h2(b_entry(t.x, q0, 2 * tg, col), b_entry(t.x, q0, 2 * tg + 1, col));
        b[1] = pack_h2(b_entry(t.x, q0, 2 * tg + 8, col), b_entry(t.x, q0, 2 * tg + 9, col));
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
        // C: (g, 2tg), (g, 2tg+1), (g+8, 2tg), (g+8, 2tg+1); rows < 12 hold the two sites
#pragma unroll
        for (int e = 0; e < 4; e++) {
          const int row = g + (e >> 1) * 8, cc = 8 * cg + 2 * tg + (e & 1);
          if (row < 12) {
            const int site = row / 6, rr = row % 6;
            yf[2 * (((q0 + site) * LCOLS + cc) * 3 + rr % 3) + (rr < 3 ? 0 : 1)] = c[e];
          }
        }
      }
    }
    __syncthreads();
  }
  if (out)
    for (int i = threadIdx.x; i < LQ * LCOLS * 3; i += blockDim.x) out[(size_t)blockIdx.x * LQ * LCOLS * 3 + i] = t.y[i];
}

size_t tile_smem(int method) {
  const size_t e = method == 0 ? sizeof(float2) : sizeof(__half2);
  return e * (LQ * 9 + LQ * LCOLS * 3) + sizeof(float2) * LQ * LCOLS * 3;
}

int launch_probe(int method, int ctas, int reps, float2 *out, cudaStream_t st) {
  const size_t sm = tile_smem(method);
  switch (method) {
    case 0:
      DD_CUDA(cudaFuncSetAttribute(k_link_alu<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_link_alu<float2><<<ctas, LTPB, sm, st>>>(reps, out);
      break;
    case 1:
      DD_CUDA(cudaFuncSetAttribute(k_link_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_link_mma<<<ctas, LTPB, sm, st>>>(reps, out);
      break;
    case 2:
      DD_CUDA(cudaFuncSetAttribute(k_link_alu<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_link_alu<__half2><<<ctas, LTPB, sm, st>>>(reps, out);
      break;
    default:
      set_error("dd_bench_link_product: method 0, 1 or 2");
      return DD_EINVAL;
  }
  return launched("link product probe");
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" int dd_bench_link_product(int method, int ctas, int reps, double *ms, double *rel_diff) {
  if (ctas < 1 || reps < 1 || !ms || method < 0 || method > 2) {
    set_error("dd_bench_link_product: bad argument");
    return DD_EINVAL;
  }
  const size_t n = (size_t)ctas * LQ * LCOLS * 3;
  float2 *out = nullptr, *ref = nullptr;
  DD_CUDA(cudaMalloc(&out, 2 * n * sizeof(float2)));
  ref = out + n;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = launch_probe(method, ctas, 1, nullptr, 0);   // warm-up
  if (rc == DD_OK) {
    cudaEventRecord(e0, 0);
    rc = launch_probe(method, ctas, reps, nullptr, 0);
    cudaEventRecord(e1, 0);
  }
  if (rc == DD_OK) rc = cuda_fail(cudaEventSynchronize(e1), "link product probe");
  float t = 0;
  if (rc == DD_OK) {
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t;
  }
  // the products of this method against the FP32 method's on the same inputs
  if (rc == DD_OK && rel_diff) {
    rc = launch_probe(method, ctas, 1, out, 0);
    if (rc == DD_OK) rc = launch_probe(0, ctas, 1, ref, 0);
    std::vector<float2> a(n), b(n);
    if (rc == DD_OK) rc = cuda_fail(cudaMemcpy(a.data(), out, n * sizeof(float2), cudaMemcpyDeviceToHost), "probe");
    if (rc == DD_OK) rc = cuda_fail(cudaMemcpy(b.data(), ref, n * sizeof(float2), cudaMemcpyDeviceToHost), "probe");
    if (rc == DD_OK) {
      double num = 0, den = 0;
      for (size_t i = 0; i < n; i++) {
        const double dx = a[i].x - b[i].x, dy = a[i].y - b[i].y;
        num = fmax(num, fabs(dx) + fabs(dy));
        den = fmax(den, fabs((double)b[i].x) + fabs((double)b[i].y));
      }
      *rel_diff = den > 0 ? num / den : 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}
