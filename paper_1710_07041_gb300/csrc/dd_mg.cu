// Two-level aggregation multigrid (the coarse-grid correction of
// DD-alpha-AMG, which the paper's Sec. 1 names as its solver; Sec. 3.1's
// Schwarz method is its fine-level smoother). The paper prints none of it;
// this is the standard form:
//   aggregates = the lattice's Schwarz blocks; N test vectors v_k;
//   P: on every aggregate a and chirality h (spins {0,1} / {2,3}) the test
//      vectors restricted to (a, h), orthonormalised by modified Gram-Schmidt
//      in the order v_1..v_N; coarse index (a, h, k); coarse vector layout
//      [aggregate][h][k] complex;
//   D_c = P^dagger D P (Galerkin), a nearest-neighbour stencil on the block
//      grid with 2N x 2N blocks: self, +mu and -mu for mu = x, y, z, t;
//   M r = P e_c + SAP(r - D P e_c), e_c ~ D_c^-1 P^dagger r by GMRES.
// Everything here computes in FP32 (the preconditioner's precision; P and
// D_c are stored in FP16); FGMRES outside keeps the FP64-class outer
// arithmetic.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "dd_mg.cuh"

namespace dd {
namespace {

constexpr int MG_TPB = 256;
__device__ __forceinline__ int colour16(const Geom &g, int b) {
  int bc[4];
  block_coords(g, b, bc);
  return (bc[0] & 1) | ((bc[1] & 1) << 1) | ((bc[2] & 1) << 2) | ((bc[3] & 1) << 3);
}

// coarse neighbour of block a in stencil direction d (0 self, 1+2mu +mu, 2+2mu -mu);
// the direction is selected by an unrolled loop so that no Geom array is
// indexed at run time (which would copy the kernel parameter to local memory)
__device__ __forceinline__ int coarse_nbr(const Geom &g, int a, int d) {
  if (d == 0) return a;
  const int mu = (d - 1) >> 1, dir = (d & 1) ? +1 : -1;
  int res = a;
#pragma unroll
  for (int m = 0; m < 4; m++)
    if (m == mu) {
      const int bcm = (a / g.bstride[m]) % g.nb[m];
      int v = bcm + dir;
      if (v < 0) v += g.nb[m];
      if (v >= g.nb[m]) v -= g.nb[m];
      res = a + (v - bcm) * g.bstride[m];
    }
  return res;
}

__device__ __forceinline__ float2 cfma_c(float2 a, float2 b, float2 acc) {  // acc += conj(a) b
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
  return acc;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {  // acc += a b
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  return acc;
}

// Per-aggregate restriction of the fine FP32 field `in` against the N basis
// fields V: out[(h * N + k)] of this CTA's aggregate, optionally only over the
// sites of one face (face = 2 mu + side, side 1 = upper; -1 = all sites).
// Returns through smem; thread t < 2N writes result t to dst[t * dst_stride].
template <int NMAX, typename SV>
__device__ void restrict_block(const Geom &g, int b, const void *V, size_t fbytes, int N, const float *in, int face,
                               float2 *dst, int dst_stride) {
  __shared__ float2 red[MG_TPB / 32][2 * NMAX];
  const int s = threadIdx.x;
  float2 acc[2 * NMAX];
#pragma unroll
  for (int q = 0; q < 2 * NMAX; q++) acc[q] = make_float2(0.f, 0.f);
  if (s < g.Vb) {
    bool take = true;
    if (face >= 0) {
      int lc[4];
      local_coords(g, s, lc);
      const int mu = face >> 1;
      take = lc[mu] == ((face & 1) ? g.bd[mu] - 1 : 0);
    }
    if (take) {
      Spinor<float> r;
      load_spinor<float, float>(in, g, b, s, r);
#pragma unroll
      for (int k = 0; k < NMAX; k++) {
        if (k < N) {
          Spinor<float> v;
          load_spinor<SV, float>((const char *)V + k * fbytes, g, b, s, v);
          float2 up = make_float2(0.f, 0.f), dn = make_float2(0.f, 0.f);
#pragma unroll
          for (int c = 0; c < 6; c++) {
            up = cfma_c(make_float2(v.c[c].re, v.c[c].im), make_float2(r.c[c].re, r.c[c].im), up);
            dn = cfma_c(make_float2(v.c[6 + c].re, v.c[6 + c].im), make_float2(r.c[6 + c].re, r.c[6 + c].im), dn);
          }
          acc[k] = up;
          acc[NMAX + k] = dn;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < 2 * NMAX; q++) {
    if ((q % NMAX) >= N) continue;
    float2 v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) red[w][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * N) {
    const int h = threadIdx.x / N, k = threadIdx.x - h * N;
    float2 t = make_float2(0.f, 0.f);
    for (int i = 0; i < nw; i++) {
      float2 u = red[i][h * NMAX + k];
      t.x += u.x;
      t.y += u.y;
    }
    dst[threadIdx.x * dst_stride] = t;
  }
  __syncthreads();
}

// restriction with the FP16 interpolation fields
template <int NMAX>
__global__ void __launch_bounds__(MG_TPB) k_restrict(Geom g, const __half *V, size_t fbytes, int N, const float *in,
                                                    float2 *out) {
  restrict_block<NMAX, __half>(g, blockIdx.x, V, fbytes, N, in, -1, out + (size_t)blockIdx.x * 2 * N, 1);
}

// Column (h', j) of D_c for aggregates coupled to colour class c16: w = D u
// with u = v_j on chirality h' of the colour-c16 aggregates. An aggregate of
// colour c16 receives its self block; one whose colour differs in exactly one
// direction bit mu receives the +mu block through its upper mu-face and the
// -mu block through its lower one. Dc layout: [a][d][col][row].
template <int NMAX>
__global__ void __launch_bounds__(MG_TPB) k_restrict_dc(Geom g, const float *V, size_t fstride, int N,
                                                       const float *w, float2 *Dc, int c16, int col) {
  const int a = blockIdx.x, diff = colour16(g, a) ^ c16;
  const int n2 = 2 * N;
  float2 *base = Dc + (size_t)a * 9 * n2 * n2;
  if (diff == 0) {
    restrict_block<NMAX, float>(g, a, V, fstride * 4, N, w, -1, base + (size_t)col * n2, 1);
  } else if ((diff & (diff - 1)) == 0) {
    const int mu = __ffs(diff) - 1;
    restrict_block<NMAX, float>(g, a, V, fstride * 4, N, w, 2 * mu + 1,
                                base + ((size_t)(1 + 2 * mu) * n2 + col) * n2, 1);
    restrict_block<NMAX, float>(g, a, V, fstride * 4, N, w, 2 * mu, base + ((size_t)(2 + 2 * mu) * n2 + col) * n2, 1);
  }
}

// u = v_j on chirality hp of the aggregates of colour c16, zero elsewhere
__global__ void k_column(Geom g, const float *vj, int hp, int c16, float *u) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  Spinor<float> v;
  load_spinor<float, float>(vj, g, b, s, v);
  const bool on = colour16(g, b) == c16;
#pragma unroll
  for (int c = 0; c < 12; c++)
    if (!on || (c / 6) != hp) v.c[c] = {0.f, 0.f};
  store_spinor<float, float>(u, g, b, s, v);
}

// x(site) = sum_k v_k(site) c[a][h(spin)][k]  (+ x when accumulate)
__global__ void k_prolong(Geom g, const __half *V, size_t fbytes, int N, const float2 *c, float *x) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  const float2 *cb = c + (size_t)b * 2 * N;
  float2 o[12];
#pragma unroll
  for (int q = 0; q < 12; q++) o[q] = make_float2(0.f, 0.f);
  for (int k = 0; k < N; k++) {
    Spinor<float> v;
    load_spinor<__half, float>((const char *)V + k * fbytes, g, b, s, v);
    const float2 cu = cb[k], cd = cb[N + k];
#pragma unroll
    for (int q = 0; q < 12; q++) o[q] = cfma(make_float2(v.c[q].re, v.c[q].im), q < 6 ? cu : cd, o[q]);
  }
  Spinor<float> out;
#pragma unroll
  for (int q = 0; q < 12; q++) out.c[q] = {o[q].x, o[q].y};
  store_spinor<float, float>(x, g, b, s, out);
}

// Per (aggregate, chirality): modified Gram-Schmidt of the N test vectors in
// order, in place (FP32 data, FP32 sums). One CTA per (aggregate, h).
__global__ void __launch_bounds__(MG_TPB) k_orthonormalise(Geom g, float *V, size_t fstride, int N) {
  __shared__ float red[MG_TPB / 32][2];
  const int b = blockIdx.x >> 1, h = blockIdx.x & 1, s = threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  // this thread's 6 components (site s, chirality h) of every vector: address helper
  auto addr = [&](int k, int c) -> float2 * {
    // F32 spinor layout: chunk = 2 complex; component c of half h = spinor component 6h + c
    const int comp = 6 * h + c;
    return (float2 *)((char *)(V + k * fstride) + (((size_t)b * 6 + comp / 2) * g.Vb + s) * 16 + (comp & 1) * 8);
  };
  auto bsum2 = [&](float2 v) {
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) {
      red[w][0] = v.x;
      red[w][1] = v.y;
    }
    __syncthreads();
    float2 t = make_float2(0.f, 0.f);
    for (int i = 0; i < nw; i++) {
      t.x += red[i][0];
      t.y += red[i][1];
    }
    __syncthreads();
    return t;
  };
  const bool act = s < g.Vb;
  for (int k = 0; k < N; k++) {
    float2 vk[6];
#pragma unroll
    for (int c = 0; c < 6; c++) vk[c] = act ? *addr(k, c) : make_float2(0.f, 0.f);
    for (int j = 0; j < k; j++) {
      float2 d = make_float2(0.f, 0.f), qj[6];
#pragma unroll
      for (int c = 0; c < 6; c++) {
        qj[c] = act ? *addr(j, c) : make_float2(0.f, 0.f);
        d = cfma_c(qj[c], vk[c], d);
      }
      d = bsum2(d);
#pragma unroll
      for (int c = 0; c < 6; c++) {
        vk[c].x -= d.x * qj[c].x - d.y * qj[c].y;
        vk[c].y -= d.x * qj[c].y + d.y * qj[c].x;
      }
    }
    float2 n2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 6; c++) n2.x += vk[c].x * vk[c].x + vk[c].y * vk[c].y;
    n2 = bsum2(n2);
    const float inv = n2.x > 0.f ? rsqrtf(n2.x) : 0.f;
    if (act)
#pragma unroll
      for (int c = 0; c < 6; c++) *addr(k, c) = make_float2(vk[c].x * inv, vk[c].y * inv);
    __syncthreads();
  }
}

// Rows of a stored coarse column, padded to a multiple of 4 so that a column
// is a whole number of 16-byte chunks (4 complex FP16 entries each).
__host__ __device__ __forceinline__ int dc_rows(int N) { return (2 * N + 3) & ~3; }

// Launch shape of the coarse apply: R = rows/4 chunk lanes times Q column
// groups, at most 256 threads.
static inline void coarse_shape(int N, int *R, int *Q) {
  *R = dc_rows(N) / 4;
  const int q = 256 / *R;
  *Q = q < 18 * N ? q : 18 * N;
}

// y = D_c (s x), s = 1 / *scale (or 1). D_c is stored as complex FP16
// [a][q = d * 2N + col][row (padded)], summed in FP32. One CTA per aggregate;
// thread t owns rows 4r..4r+3 (r = t mod R) of the columns q = t / R + k Q and
// loads them as one 16-byte chunk per column; the Q column groups' partial
// sums are added in shared memory in a fixed order. With NPRE > 0 a thread
// issues all its (at most NPRE) chunk loads before gathering x, so the
// operator stream overlaps the gather. With vnext != null the CTA also stores
// its own part of s x there (the next Krylov basis vector).
template <int NPRE>
__global__ void __launch_bounds__(256) k_coarse_apply(Geom g, const __half2 *__restrict__ Dc, int N, int R, int Q,
                                                      const float2 *__restrict__ x, float2 *y, const float *scale,
                                                      float2 *vnext, const int *done) {
  if (done && *done) return;
  extern __shared__ float2 sm[];   // xs[9 * 2N], then red[Q][rows]
  const int a = blockIdx.x, n2 = 2 * N, np = 4 * R, ncol = 9 * n2;
  const int r = threadIdx.x % R, qg = threadIdx.x / R;
  const uint4 *D = reinterpret_cast<const uint4 *>(Dc + (size_t)a * ncol * np);
  uint4 pre[NPRE > 0 ? NPRE : 1];
#pragma unroll
  for (int k = 0; k < NPRE; k++) {
    const int q = qg + k * Q;
    pre[k] = q < ncol ? __ldcs(D + (size_t)q * R + r) : make_uint4(0, 0, 0, 0);
  }
  float2 *xs = sm, *red = sm + ncol;
  const float sc = scale ? 1.f / *scale : 1.f;
  for (int q = threadIdx.x; q < ncol; q += blockDim.x) {
    const int d = q / n2, c = q - d * n2;
    int na = coarse_nbr(g, a, d);
    DD_CHECK_INDEX(na, g.nblocks);
    const float2 v = x[(size_t)na * n2 + c];
    xs[q] = make_float2(v.x * sc, v.y * sc);
  }
  __syncthreads();
  if (vnext)
    for (int row = threadIdx.x; row < n2; row += blockDim.x) vnext[(size_t)a * n2 + row] = xs[row];
  float2 acc[4];
#pragma unroll
  for (int k = 0; k < 4; k++) acc[k] = make_float2(0.f, 0.f);
  if (NPRE > 0) {
#pragma unroll
    for (int k = 0; k < NPRE; k++) {
      const int q = qg + k * Q;
      if (q < ncol) {
        const float2 xq = xs[q];
        const __half2 *h = reinterpret_cast<const __half2 *>(&pre[k]);
#pragma unroll
        for (int c = 0; c < 4; c++) acc[c] = cfma(__half22float2(h[c]), xq, acc[c]);
      }
    }
  } else {
#pragma unroll 4
    for (int q = qg; q < ncol; q += Q) {
      const uint4 c4 = __ldcs(D + (size_t)q * R + r);
      const float2 xq = xs[q];
      const __half2 *h = reinterpret_cast<const __half2 *>(&c4);
#pragma unroll
      for (int c = 0; c < 4; c++) acc[c] = cfma(__half22float2(h[c]), xq, acc[c]);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; k++) red[qg * np + 4 * r + k] = acc[k];
  __syncthreads();
  for (int row = threadIdx.x; row < n2; row += blockDim.x) {
    float2 t = make_float2(0.f, 0.f);
    for (int q = 0; q < Q; q++) {
      t.x += red[q * np + row].x;
      t.y += red[q * np + row].y;
    }
    y[(size_t)a * n2 + row] = t;
  }
}

// FP32 [a][q][2N] -> FP16 [a][q][rows], padding rows zero
__global__ void k_dc_to_half(const float2 *in, __half2 *out, size_t ncols, int n2, int np) {
  const size_t n = ncols * np;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const size_t col = e / np;
    const int row = (int)(e - col * np);
    const float2 v = row < n2 ? in[col * n2 + row] : make_float2(0.f, 0.f);
    out[e] = __floats2half2_rn(v.x, v.y);
  }
}

// ---------------------------------------------------------- coarse GMRES
// GMRES(k) on D_c with one cycle of at most `kmax` steps from x = 0 and the
// control (Givens rotations, convergence test) on the device, so a coarse
// solve needs no host synchronisation and can be captured in a CUDA graph.
// Three launches per step: (1) w' = D_c v_j, v_j = w / h_{j,j-1} formed on
// the fly; (2) the projections H[i][j] = <v_i, w'>; (3) w' -= sum_i H[i][j]
// v_i with its norm, then the Givens update. Kernels (2) and (3) finish with
// the last CTA summing all CTAs' partials in a fixed order (deterministic).
struct CgState {
  int j, done, steps;
  unsigned count;          // CTAs finished in the current reduction
  float bnorm, tol, hn;
  float2 H[65 * 64];       // H[i * 64 + j]
  float2 g[65];
  float cs[64];
  float2 sn[64];
  float2 y[64];
};

constexpr int CG_GRID = 1024;   // maximum CTAs of the start and final update
constexpr int CG_EPT = 4;       // float4 per thread in a projection
constexpr int CG_ROWS = 4;      // basis vectors per projection CTA

static inline int cg_grid(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < CG_GRID ? (b ? b : 1) : CG_GRID);
}
// CTAs per projection row; CTAs of the update (one float4 per thread)
static inline int cg_chunks(size_t n) { return (int)((n / 2 + 256 * CG_EPT - 1) / (256 * CG_EPT)); }
static inline int cg_upd_grid(size_t n) { return (int)((n / 2 + 255) / 256); }
static inline int cg_partials(size_t n) { return cg_upd_grid(n) > CG_GRID ? cg_upd_grid(n) : CG_GRID; }

// is this CTA the last of the grid to arrive? (after its partial is stored)
__device__ __forceinline__ bool last_cta(unsigned *count, unsigned total) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(count, 1u) == total - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// sum over a 256-thread CTA in a fixed order; every thread gets the result.
// The coarse solve reduces in FP32 throughout: FP64 instructions issue at a
// small fraction of the FP32 rate here, and the coarse solve is an FP32
// inner solve of a flexible outer method.
__device__ __forceinline__ float cta_sum(float v) {
  __shared__ float red[8];
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < 8; q++) t += red[q];
  return t;
}

// sum of partial[0 .. P) by a 256-thread CTA, fixed order
__device__ __forceinline__ float cta_sum_partials(const float *partial, int P) {
  float t = 0.f;
  for (int b = threadIdx.x; b < P; b += 256) t += __ldcg(partial + b);
  return cta_sum(t);
}

// H[i][j] = <v_i, w> for i <= j. CTA (c, y) covers the rows i = CG_ROWS y ..
// CG_ROWS y + CG_ROWS - 1 on float4 (two complex) indices
// c * 256 * CG_EPT + t + 256 u, u < CG_EPT; all its loads are issued together.
__global__ void __launch_bounds__(256) k_cg_proj(const float2 *Vc, size_t n, const float2 *w, float2 *partial,
                                                 int chunks, CgState *st) {
  if (st->done) return;
  __shared__ float2 red[8][CG_ROWS];
  const int k = st->j + 1, i0 = blockIdx.y * CG_ROWS;
  const size_t n4 = n / 2;
  const float4 *w4 = reinterpret_cast<const float4 *>(w);
  const size_t e0 = (size_t)blockIdx.x * 256 * CG_EPT + threadIdx.x;
  float4 ww[CG_EPT], vv[CG_ROWS][CG_EPT];
#pragma unroll
  for (int u = 0; u < CG_EPT; u++) {
    const size_t e = e0 + 256 * u;
    ww[u] = e < n4 ? w4[e] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < CG_ROWS; q++)
      vv[q][u] = (e < n4 && i0 + q < k) ? reinterpret_cast<const float4 *>(Vc + (size_t)(i0 + q) * n)[e]
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < CG_ROWS; q++) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < CG_EPT; u++) {
      acc = cfma_c(make_float2(vv[q][u].x, vv[q][u].y), make_float2(ww[u].x, ww[u].y), acc);
      acc = cfma_c(make_float2(vv[q][u].z, vv[q][u].w), make_float2(ww[u].z, ww[u].w), acc);
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = acc;
  }
  __syncthreads();
  if (threadIdx.x < CG_ROWS && i0 + (int)threadIdx.x < k) {
    float2 t = make_float2(0.f, 0.f);
    for (int wq = 0; wq < 8; wq++) {
      t.x += red[wq][threadIdx.x].x;
      t.y += red[wq][threadIdx.x].y;
    }
    partial[(size_t)(i0 + threadIdx.x) * chunks + blockIdx.x] = t;
  }
  if (last_cta(&st->count, gridDim.x * gridDim.y)) {
    // warp w sums rows i = w, w + 8, ...; lane l the partials l, l + 32, ...
    const int lane = threadIdx.x & 31, j = st->j;
    for (int q = threadIdx.x >> 5; q < k; q += 8) {
      float2 t = make_float2(0.f, 0.f);
      for (int b = lane; b < chunks; b += 32) {
        const float2 pv = __ldcg(&partial[(size_t)q * chunks + b]);
        t.x += pv.x;
        t.y += pv.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
        t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
      }
      if (lane == 0) st->H[q * 64 + j] = t;
    }
    if (threadIdx.x == 0) st->count = 0;
  }
}

// finish step j: apply the earlier rotations to column j of H, form the new
// one, update g and test convergence. Run by one CTA (the last to arrive);
// the column and the rotations are staged in shared memory. The rotations
// are FP32 like the coarse vectors (FP64 runs at a small fraction of the
// FP32 rate here and this chain is serial).
__device__ void cg_givens(float n2, CgState *st, int kmax) {
  __shared__ float2 col[65], sn[64];
  __shared__ float cs[64];
  const int j = st->j;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = st->H[i * 64 + j];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cs[i] = st->cs[i];
    sn[i] = st->sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float hn = sqrtf(n2 > 0.f ? n2 : 0.f);
    for (int i = 0; i < j; i++) {
      const float2 a = col[i], c = col[i + 1], s = sn[i];
      const float ci = cs[i];
      // a' = cs a + sn c ; c' = -conj(sn) a + cs c
      col[i] = make_float2(ci * a.x + s.x * c.x - s.y * c.y, ci * a.y + s.x * c.y + s.y * c.x);
      col[i + 1] = make_float2(-(s.x * a.x + s.y * a.y) + ci * c.x, -(s.x * a.y - s.y * a.x) + ci * c.y);
    }
    const float2 a = col[j];
    const float aa = sqrtf(a.x * a.x + a.y * a.y), rr = sqrtf(aa * aa + hn * hn);
    float c;
    float2 s;
    if (aa == 0.f) {
      c = 0.f;
      s = make_float2(1.f, 0.f);
    } else {
      const float inv = 1.f / (aa * rr);
      c = aa * aa * inv;
      s = make_float2(a.x * hn * inv, a.y * hn * inv);
    }
    st->cs[j] = c;
    st->sn[j] = s;
    col[j] = make_float2(c * a.x + s.x * hn, c * a.y + s.y * hn);
    const float2 gj = st->g[j];
    const float2 g1 = make_float2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    st->g[j + 1] = g1;
    st->g[j] = make_float2(c * gj.x, c * gj.y);
    st->hn = hn;
    st->steps = j + 1;
    const float est = sqrtf(g1.x * g1.x + g1.y * g1.y);
    if (est <= st->tol * st->bnorm || hn == 0.f || j + 1 >= kmax) st->done = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) st->H[i * 64 + j] = col[i];
  __syncthreads();
  if (threadIdx.x == 0) st->j = j + 1;
}

// w -= sum_{i<=j} H[i][j] v_i, then |w|^2 and the Givens step (last CTA).
// Thread t of CTA c owns float4 (two complex numbers) c * 256 + t.
__global__ void __launch_bounds__(256) k_cg_update_w(const float2 *Vc, size_t n, float2 *w, float *partial,
                                                     CgState *st, int kmax) {
  if (st->done) return;
  __shared__ float2 hs[64];
  const int k = st->j + 1;
  for (int i = threadIdx.x; i < k; i += blockDim.x) hs[i] = st->H[i * 64 + st->j];
  __syncthreads();
  const size_t n4 = n / 2, e = (size_t)blockIdx.x * 256 + threadIdx.x;
  float nrm = 0.f;
  if (e < n4) {
    float4 *w4 = reinterpret_cast<float4 *>(w);
    float4 we = w4[e];
#pragma unroll 8
    for (int i = 0; i < k; i++) {
      const float4 v = reinterpret_cast<const float4 *>(Vc + (size_t)i * n)[e];
      const float2 h = hs[i];
      we.x -= h.x * v.x - h.y * v.y;
      we.y -= h.x * v.y + h.y * v.x;
      we.z -= h.x * v.z - h.y * v.w;
      we.w -= h.x * v.w + h.y * v.z;
    }
    w4[e] = we;
    nrm = we.x * we.x + we.y * we.y + we.z * we.z + we.w * we.w;
  }
  const float tot = cta_sum(nrm);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
  if (last_cta(&st->count, gridDim.x)) {
    const float t = cta_sum_partials(partial, gridDim.x);
    if (threadIdx.x == 0) st->count = 0;
    cg_givens(t, st, kmax);
  }
}

// start: |b|^2 partials, then (last CTA) the state; v_0 = b / |b| is formed
// by the first apply
__global__ void __launch_bounds__(256) k_cg_start(const float2 *b, size_t n, float *partial, CgState *st, float tol) {
  float nrm = 0.f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    nrm = fmaf(b[e].x, b[e].x, fmaf(b[e].y, b[e].y, nrm));
  nrm = cta_sum(nrm);
  if (threadIdx.x == 0) partial[blockIdx.x] = nrm;
  if (last_cta(&st->count, gridDim.x)) {
    const float t = cta_sum_partials(partial, gridDim.x);
    for (int i = threadIdx.x; i < 65; i += blockDim.x) st->g[i] = make_float2(0.f, 0.f);
    __syncthreads();
    if (threadIdx.x == 0) {
      const float bn = sqrtf(t > 0.f ? t : 0.f);
      st->count = 0;
      st->bnorm = bn;
      st->tol = tol;
      st->j = 0;
      st->steps = 0;
      st->done = bn == 0.f;
      st->g[0] = make_float2(bn, 0.f);
      st->hn = bn;
    }
  }
}

// back substitution R y = g, column by column, R staged in shared memory as a
// packed upper triangle (column l holds rows 0..l at l (l + 1) / 2) and the
// reciprocals of its diagonal formed in parallel first
__global__ void __launch_bounds__(64) k_cg_solve(CgState *st) {
  __shared__ float2 R[64 * 65 / 2], t[64], rd[64];
  const int k = st->steps, tri = k * (k + 1) / 2;
  for (int p = threadIdx.x; p < tri; p += blockDim.x) {
    int l = (int)((sqrtf(8.f * p + 1.f) - 1.f) * 0.5f);   // column of packed index p
    while (l * (l + 1) / 2 > p) l--;
    while ((l + 1) * (l + 2) / 2 <= p) l++;
    R[p] = st->H[(p - l * (l + 1) / 2) * 64 + l];
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    t[i] = st->g[i];
    const float2 d = st->H[i * 64 + i];
    const float dd = d.x * d.x + d.y * d.y;
    rd[i] = dd > 0.f ? make_float2(d.x / dd, -d.y / dd) : make_float2(0.f, 0.f);   // 1 / d
  }
  __syncthreads();
  for (int l = k - 1; l >= 0; l--) {
    const float2 tl = t[l], r = rd[l];
    const float2 yl = make_float2(tl.x * r.x - tl.y * r.y, tl.x * r.y + tl.y * r.x);
    if (threadIdx.x == 0) st->y[l] = yl;
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
      const float2 h = R[l * (l + 1) / 2 + i];
      t[i].x -= h.x * yl.x - h.y * yl.y;
      t[i].y -= h.x * yl.y + h.y * yl.x;
    }
    __syncthreads();
  }
}

// x = sum_i y_i v_i
__global__ void __launch_bounds__(256) k_cg_update(const float2 *Vc, size_t n, float2 *x, const CgState *st) {
  __shared__ float2 ys[64];
  const int k = st->steps;
  for (int i = threadIdx.x; i < k; i += blockDim.x) ys[i] = st->y[i];
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int i = 0; i < k; i++) acc = cfma(ys[i], Vc[i * n + e], acc);
    x[e] = acc;
  }
}

// fine FP32 fields: y = a - b
__global__ void k_sub(const float4 *a, const float4 *b, float4 *y, size_t n4) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
    const float4 u = a[e], v = b[e];
    y[e] = make_float4(u.x - v.x, u.y - v.y, u.z - v.z, u.w - v.w);
  }
}
// y = (a + b) * s
__global__ void k_add_scale(const float4 *a, const float4 *b, float4 *y, float s, size_t n4) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
    const float4 u = a[e], v = b[e];
    y[e] = make_float4((u.x + v.x) * s, (u.y + v.y) * s, (u.z + v.z) * s, (u.w + v.w) * s);
  }
}

}  // namespace

// ---------------------------------------------------------------- MgWork
MgWork::~MgWork() {
  for (auto &kv : graphs) cudaGraphExecDestroy(kv.second.first);
  void *p[] = {Vc, w, w2, cb, ce, xf, rf, tf, tin, tout, partial, pnorm, st};
  for (void *q : p)
    if (q) cudaFree(q);
}

int MgWork::init(const Mg *mg) {
  const Geom &g = mg->op->lat->g;
  nc = (size_t)g.nblocks * 2 * mg->N;
  const size_t f32 = (size_t)g.V * 24 * 4, fp = (size_t)g.V * spinor_site_bytes(mg->op->prec);
  const int kmax = mg->p.coarse_max_iter;
  bool ok = cudaMalloc(&Vc, sizeof(float2) * nc * (kmax + 1)) == cudaSuccess &&
            cudaMalloc(&w, sizeof(float2) * nc) == cudaSuccess && cudaMalloc(&w2, sizeof(float2) * nc) == cudaSuccess &&
            cudaMalloc(&cb, sizeof(float2) * nc) == cudaSuccess &&
            cudaMalloc(&ce, sizeof(float2) * nc) == cudaSuccess && cudaMalloc(&xf, f32) == cudaSuccess &&
            cudaMalloc(&rf, f32) == cudaSuccess && cudaMalloc(&tf, f32) == cudaSuccess &&
            cudaMalloc(&tin, fp) == cudaSuccess && cudaMalloc(&tout, fp) == cudaSuccess &&
            cudaMalloc(&partial, sizeof(float2) * cg_chunks(nc) * 65) == cudaSuccess &&
            cudaMalloc(&pnorm, sizeof(float) * cg_partials(nc)) == cudaSuccess &&
            cudaMalloc(&st, sizeof(CgState)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    set_error("mg: out of device memory for the coarse-solve workspace");
    return DD_ENOMEM;
  }
  return cuda_fail(cudaMemset(st, 0, sizeof(CgState)), "mg workspace");   // reduction counter = 0
}

size_t MgWork::bytes(const Geom &g, int prec, int N, int kmax) {
  const size_t nc = (size_t)g.nblocks * 2 * N;
  return sizeof(float2) * nc * (kmax + 5) + (size_t)g.V * 24 * (4 * 3 + 2 * real_bytes(prec)) +
         sizeof(float2) * cg_chunks(nc) * 65 + sizeof(float) * cg_partials(nc) + sizeof(CgState);
}

// ------------------------------------------------------------- operations
static int restrict_launch(const Mg *mg, const float *in, float2 *out, cudaStream_t st) {
  const Geom &g = mg->op->lat->g;
  const size_t fs = (size_t)g.V * 24;
  const int tpb = g.Vb > MG_TPB ? 0 : MG_TPB;
  if (!tpb) {
    set_error("mg: aggregates of more than %d sites are not supported", MG_TPB);
    return DD_EINVAL;
  }
  const size_t fb = fs * sizeof(__half);
  if (mg->N <= 8) k_restrict<8><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->Vh, fb, mg->N, in, out);
  else if (mg->N <= 16) k_restrict<16><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->Vh, fb, mg->N, in, out);
  else k_restrict<32><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->Vh, fb, mg->N, in, out);
  return launched("k_restrict");
}

int mg_restrict(const Mg *mg, const float *in, float2 *out, cudaStream_t st) { return restrict_launch(mg, in, out, st); }

int mg_prolong(const Mg *mg, const float2 *c, float *out, cudaStream_t st) {
  const Geom &g = mg->op->lat->g;
  k_prolong<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>(g, mg->Vh, (size_t)g.V * 24 * sizeof(__half), mg->N, c,
                                                            out);
  return launched("k_prolong");
}

static int coarse_apply_launch(const Mg *mg, const float2 *x, float2 *y, const float *scale, float2 *vnext,
                               const int *done, cudaStream_t st) {
  const Geom &g = mg->op->lat->g;
  int R, Q;
  coarse_shape(mg->N, &R, &Q);
  const size_t shm = sizeof(float2) * (18 * (size_t)mg->N + (size_t)Q * 4 * R);
  const int per = (18 * mg->N + Q - 1) / Q;   // chunks per thread
  const dim3 grid(g.nblocks), blk(R * Q);
  if (per <= 4) k_coarse_apply<4><<<grid, blk, shm, st>>>(g, mg->Dc, mg->N, R, Q, x, y, scale, vnext, done);
  else if (per <= 8) k_coarse_apply<8><<<grid, blk, shm, st>>>(g, mg->Dc, mg->N, R, Q, x, y, scale, vnext, done);
  else if (per <= 12) k_coarse_apply<12><<<grid, blk, shm, st>>>(g, mg->Dc, mg->N, R, Q, x, y, scale, vnext, done);
  else k_coarse_apply<0><<<grid, blk, shm, st>>>(g, mg->Dc, mg->N, R, Q, x, y, scale, vnext, done);
  return launched("k_coarse_apply");
}

int mg_coarse_apply(const Mg *mg, const float2 *x, float2 *y, cudaStream_t st) {
  return coarse_apply_launch(mg, x, y, nullptr, nullptr, nullptr, st);
}

// e = GMRES_kmax(D_c, b) from 0 (device-side control, 3 launches per step)
int mg_coarse_solve(const Mg *mg, MgWork &W, const float2 *b, float2 *e, cudaStream_t st) {
  const size_t n = W.nc;
  const int kmax = mg->p.coarse_max_iter, grid = cg_grid(n);
  CgState *cs = (CgState *)W.st;
  k_cg_start<<<grid, 256, 0, st>>>(b, n, W.pnorm, cs, (float)mg->p.coarse_tol);
  DD_LAUNCHED();
  const float2 *src = b;      // v_j = src / hn
  float2 *wbuf[2] = {W.w, W.w2};
  int rc;
  for (int j = 0; j < kmax; j++) {
    float2 *wj = wbuf[j & 1];
    if ((rc = coarse_apply_launch(mg, src, wj, &cs->hn, W.Vc + (size_t)j * n, &cs->done, st))) return rc;
    k_cg_proj<<<dim3(cg_chunks(n), (j + CG_ROWS) / CG_ROWS), 256, 0, st>>>(W.Vc, n, wj, W.partial, cg_chunks(n), cs);
    DD_LAUNCHED();
    k_cg_update_w<<<cg_upd_grid(n), 256, 0, st>>>(W.Vc, n, wj, W.pnorm, cs, kmax);
    DD_LAUNCHED();
    src = wj;
  }
  k_cg_solve<<<1, 64, 0, st>>>(cs);
  DD_LAUNCHED();
  k_cg_update<<<grid, 256, 0, st>>>(W.Vc, n, e, cs);
  return launched("k_cg_update");
}

int mg_sub(const float *a, const float *b, float *y, size_t n_floats, cudaStream_t st) {
  k_sub<<<1024, 256, 0, st>>>((const float4 *)a, (const float4 *)b, (float4 *)y, n_floats / 4);
  return launched("k_sub");
}
int mg_add_scale(const float *a, const float *b, float *y, float s, size_t n_floats, cudaStream_t st) {
  k_add_scale<<<1024, 256, 0, st>>>((const float4 *)a, (const float4 *)b, (float4 *)y, s, n_floats / 4);
  return launched("k_add_scale");
}

// M r: x = scale * (P e_c + SAP(r - D P e_c)), e_c ~ D_c^-1 P^dagger r. r and x: FP32 fields.
static int mg_enqueue(const Mg *mg, MgWork &W, const float *r, float *x, cudaStream_t st, float scale) {
  const Op *op = mg->op;
  const Geom &g = op->lat->g;
  const size_t nf = (size_t)g.V * 24;
  int rc;
  if ((rc = mg_restrict(mg, r, W.cb, st))) return rc;
  if ((rc = mg_coarse_solve(mg, W, W.cb, W.ce, st))) return rc;
  if ((rc = mg_prolong(mg, W.ce, W.xf, st))) return rc;
  if ((rc = launch_dirac(g, op->f32, W.xf, W.tf, 1, st))) return rc;
  if ((rc = mg_sub(r, W.tf, W.rf, nf, st))) return rc;   // r1 = r - D x
  dd_sap_params sp = mg->p.smoother;
  sp.x_is_zero = 1;
  if (op->prec == DD_F32) {
    if ((rc = launch_sap(g, op->fp, sp, W.rf, W.tf, 1, st))) return rc;
  } else {
    if ((rc = launch_convert_field(g, DD_F32, W.rf, op->prec, W.tin, 1, 1.0, st))) return rc;
    if ((rc = launch_sap(g, op->fp, sp, W.tin, W.tout, 1, st))) return rc;
    if ((rc = launch_convert_field(g, op->prec, W.tout, DD_F32, W.tf, 1, 1.0, st))) return rc;
  }
  return mg_add_scale(W.xf, W.tf, x, scale, nf, st);
}

// A preconditioner application is about 3 kmax + 10 launches, most of them
// small (coarse vectors of 2N complex numbers per aggregate), so from the
// second application on with the same (r, x, scale) it runs as one CUDA graph
// captured on that call. The first application of a workspace runs eagerly,
// so that the autotuner has chosen the fine-grid kernels' variants before any
// capture. DD_MG_GRAPHS=0 disables the graphs; a stream under capture by the
// caller, or the legacy stream, gets the launches directly.
int mg_apply(const Mg *mg, MgWork &W, const float *r, float *x, cudaStream_t st, float scale) {
  NvtxRange range("dd:mg_apply");
  const char *env = getenv("DD_MG_GRAPHS");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if ((env && env[0] == '0') || cap != cudaStreamCaptureStatusNone || st == 0 || !W.warm) {
    W.warm = true;
    return mg_enqueue(mg, W, r, x, st, scale);
  }
  uint32_t sbits;
  memcpy(&sbits, &scale, 4);
  const std::string key = std::to_string((uintptr_t)r) + ":" + std::to_string((uintptr_t)x) + ":" +
                          std::to_string(sbits);
  auto it = W.graphs.find(key);
  if (it != W.graphs.end()) {
    count_launches((int)it->second.second);
    return cuda_fail(cudaGraphLaunch(it->second.first, st), "mg graph launch");
  }
  cudaGraph_t graph = nullptr;
  DD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = mg_enqueue(mg, W, r, x, st, scale);
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "mg graph capture");
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "mg graph instantiate");
  if (W.graphs.size() >= 128) {   // bounded: start over when full
    for (auto &kv : W.graphs) cudaGraphExecDestroy(kv.second.first);
    W.graphs.clear();
  }
  W.graphs[key] = {exec, nodes};
  return cuda_fail(cudaGraphLaunch(exec, st), "mg graph launch");
}

// ------------------------------------------------------------------ setup
static int build_coarse(Mg *mg, cudaStream_t st) {
  const Op *op = mg->op;
  const Geom &g = op->lat->g;
  const size_t fs = (size_t)g.V * 24;
  const int N = mg->N, n2 = 2 * N;
  float *u = nullptr, *wv = nullptr;
  float2 *dcf = nullptr;   // FP32 coarse operator while it is assembled
  const size_t ndc = (size_t)g.nblocks * 9 * n2 * n2;
  DD_CUDA(cudaMalloc(&u, fs * 4));
  if (cudaMalloc(&wv, fs * 4) != cudaSuccess || cudaMalloc(&dcf, sizeof(float2) * ndc) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(u);
    cudaFree(wv);
    set_error("mg: out of device memory");
    return DD_ENOMEM;
  }
  int rc = cuda_fail(cudaMemsetAsync(dcf, 0, sizeof(float2) * ndc, st), "memset");
  for (int c16 = 0; c16 < 16 && rc == DD_OK; c16++)
    for (int col = 0; col < n2 && rc == DD_OK; col++) {
      const int hp = col / N, j = col - hp * N;
      k_column<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>(g, mg->V + j * fs, hp, c16, u);
      if ((rc = launched("k_column"))) break;
      if ((rc = launch_dirac(g, op->f32, u, wv, 1, st))) break;
      if (N <= 8) k_restrict_dc<8><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N, wv, dcf, c16, col);
      else if (N <= 16) k_restrict_dc<16><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N, wv, dcf, c16, col);
      else k_restrict_dc<32><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N, wv, dcf, c16, col);
      rc = launched("k_restrict_dc");
    }
  if (rc == DD_OK) {
    k_dc_to_half<<<1024, 256, 0, st>>>(dcf, mg->Dc, (size_t)g.nblocks * 9 * n2, n2, dc_rows(N));
    rc = launched("k_dc_to_half");
  }
  if (rc == DD_OK) rc = cuda_fail(cudaStreamSynchronize(st), "mg setup");
  cudaFree(u);
  cudaFree(wv);
  cudaFree(dcf);
  return rc;
}

int mg_setup(Mg *mg, const double *tv_host, cudaStream_t st) {
  const Op *op = mg->op;
  const Geom &g = op->lat->g;
  const size_t fs = (size_t)g.V * 24;
  const int N = mg->N;
  double *canon = nullptr, *nrm = nullptr;
  void *pin = nullptr, *pout = nullptr;
  DD_CUDA(cudaMalloc(&canon, fs * 8));
  int rc = DD_OK;
  Blas bl;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((rc = bl.init(sms))) {
    cudaFree(canon);
    return rc;
  }
  if (cudaMalloc(&nrm, sizeof(double)) != cudaSuccess) rc = DD_ENOMEM;
  if (cudaMalloc(&pin, fs * real_bytes(op->prec)) != cudaSuccess ||
      cudaMalloc(&pout, fs * real_bytes(op->prec)) != cudaSuccess)
    rc = DD_ENOMEM;
  const double sigma = std::sqrt(24.0 * (double)g.V);
  for (int k = 0; k < N && rc == DD_OK; k++) {
    float *vk = mg->V + k * fs;
    rc = cuda_fail(cudaMemcpyAsync(canon, tv_host + k * fs, fs * 8, cudaMemcpyHostToDevice, st), "mg upload");
    if (rc) break;
    // smoothing v <- SAP(v), normalised to unit RMS entries (SAP is homogeneous)
    if ((rc = launch_pack(g, op->prec, canon, pin, 1, 1.0, st))) break;
    for (int it = 0; it < mg->p.setup_iters && rc == DD_OK; it++) {
      dd_sap_params sp = mg->p.smoother;
      sp.x_is_zero = 1;
      if ((rc = launch_sap(g, op->fp, sp, pin, pout, 1, st))) break;
      if ((rc = launch_unpack(g, op->prec, pout, canon, 1, 1.0, st))) break;
      if ((rc = bl.norm2(canon, fs / 2, nrm, st))) break;
      double n2 = 0;
      if ((rc = cuda_fail(cudaMemcpyAsync(&n2, nrm, sizeof(double), cudaMemcpyDeviceToHost, st), "mg norm"))) break;
      if ((rc = cuda_fail(cudaStreamSynchronize(st), "mg norm"))) break;
      const double s = n2 > 0 ? sigma / std::sqrt(n2) : 1.0;
      if ((rc = launch_pack(g, op->prec, canon, pin, 1, s, st))) break;
    }
    if (rc) break;
    if ((rc = launch_convert_field(g, op->prec, pin, DD_F32, vk, 1, 1.0, st))) break;
  }
  cudaFree(canon);
  cudaFree(nrm);
  cudaFree(pin);
  cudaFree(pout);
  if (rc) return rc;
  k_orthonormalise<<<2 * g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N);
  if ((rc = launched("k_orthonormalise"))) return rc;
  // The interpolation is kept in FP16 (restriction and prolongation read all
  // N fields per application). The FP32 copy is rounded the same way before
  // the coarse operator is assembled from it, so D_c = P^dagger D P holds
  // for the stored P.
  for (int k = 0; k < N && rc == DD_OK; k++) {
    float *vk = mg->V + k * fs;
    __half *hk = mg->Vh + k * fs;
    if ((rc = launch_convert_field(g, DD_F32, vk, DD_F16, hk, 1, 1.0, st))) break;
    rc = launch_convert_field(g, DD_F16, hk, DD_F32, vk, 1, 1.0, st);
  }
  if (rc == DD_OK) rc = build_coarse(mg, st);
  if (rc == DD_OK) {   // the FP32 copy is needed by the set-up only
    cudaFree(mg->V);
    mg->V = nullptr;
  }
  return rc;
}

}  // namespace dd

using namespace dd;

extern "C" {

int dd_create_mg(dd_op_t opp, const dd_mg_params *p, const double *tv_host, dd_mg_t *out) {
  Op *op = (Op *)opp;
  if (!op || op->magic != 0x4f505231 || !p || !tv_host || !out || p->n_vectors < 1 || p->n_vectors > 32 ||
      p->setup_iters < 0 || p->coarse_max_iter < 1 || p->coarse_max_iter > 64 || !(p->coarse_tol >= 0) ||
      p->smoother.sweeps < 1 || p->smoother.mr_steps < 0) {
    set_error("dd_create_mg: bad argument (1 <= n_vectors <= 32, 1 <= coarse_max_iter <= 64)");
    return DD_EINVAL;
  }
  const Geom &g = op->lat->g;
  if (g.Vb > MG_TPB) {
    set_error("dd_create_mg: aggregates (Schwarz blocks) of more than %d sites are not supported", MG_TPB);
    return DD_EINVAL;
  }
  if (op->prec == DD_F16N) {
    set_error("dd_create_mg: operators with DD_F16N storage are not supported");
    return DD_EINVAL;
  }
  Mg *mg = new (std::nothrow) Mg;
  if (!mg) return DD_ENOMEM;
  mg->magic = MAGIC_MG;
  mg->op = op;
  mg->p = *p;
  mg->N = p->n_vectors;
  const size_t n2 = 2 * (size_t)mg->N;
  if (cudaMalloc(&mg->V, (size_t)g.V * 24 * 4 * mg->N) != cudaSuccess ||
      cudaMalloc(&mg->Vh, (size_t)g.V * 24 * 2 * mg->N) != cudaSuccess ||
      cudaMalloc(&mg->Dc, sizeof(__half2) * (size_t)g.nblocks * 9 * n2 * dc_rows(mg->N)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(mg->V);
    cudaFree(mg->Vh);
    delete mg;
    set_error("dd_create_mg: out of device memory");
    return DD_ENOMEM;
  }
  int rc = mg->work.init(mg);
  if (rc == DD_OK) rc = mg_setup(mg, tv_host, 0);
  if (rc) {
    cudaFree(mg->V);
    cudaFree(mg->Vh);
    cudaFree(mg->Dc);
    delete mg;
    return rc;
  }
  op->refs++;
  *out = (dd_mg_t)mg;
  return DD_OK;
}

static Mg *as_mg(dd_mg_t h) {
  Mg *mg = (Mg *)h;
  return (mg && mg->magic == MAGIC_MG) ? mg : nullptr;
}

int dd_mg_restrict(dd_mg_t h, const void *fine, void *coarse, void *stream) {
  Mg *mg = as_mg(h);
  if (!mg || !fine || !coarse) {
    set_error("dd_mg_restrict: bad argument");
    return DD_EINVAL;
  }
  return mg_restrict(mg, (const float *)fine, (float2 *)coarse, (cudaStream_t)stream);
}

int dd_mg_prolong(dd_mg_t h, const void *coarse, void *fine, void *stream) {
  Mg *mg = as_mg(h);
  if (!mg || !fine || !coarse) {
    set_error("dd_mg_prolong: bad argument");
    return DD_EINVAL;
  }
  return mg_prolong(mg, (const float2 *)coarse, (float *)fine, (cudaStream_t)stream);
}

int dd_mg_coarse_apply(dd_mg_t h, const void *in, void *out, void *stream) {
  Mg *mg = as_mg(h);
  if (!mg || !in || !out || in == out) {
    set_error("dd_mg_coarse_apply: bad argument");
    return DD_EINVAL;
  }
  return mg_coarse_apply(mg, (const float2 *)in, (float2 *)out, (cudaStream_t)stream);
}

int dd_mg_precondition(dd_mg_t h, const void *r, void *x, void *stream) {
  Mg *mg = as_mg(h);
  if (!mg || !r || !x || r == x) {
    set_error("dd_mg_precondition: bad argument");
    return DD_EINVAL;
  }
  return mg_apply(mg, mg->work, (const float *)r, (float *)x, (cudaStream_t)stream);
}

size_t dd_mg_coarse_length(dd_mg_t h) {
  Mg *mg = as_mg(h);
  return mg ? (size_t)mg->op->lat->g.nblocks * 2 * mg->N : 0;
}

}  // extern "C"

namespace dd {
void destroy_mg(void *h) {
  Mg *mg = (Mg *)h;
  cudaFree(mg->V);
  cudaFree(mg->Vh);
  cudaFree(mg->Dc);
  mg->magic = 0;
  Op *op = mg->op;
  delete mg;
  release_op(op);
}
}  // namespace dd
