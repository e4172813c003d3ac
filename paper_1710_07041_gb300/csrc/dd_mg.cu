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
// Everything here works in FP32 (the preconditioner's precision); FGMRES
// outside keeps the FP64/double-float outer arithmetic.
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

// coarse neighbour of block a in stencil direction d (0 self, 1+2mu +mu, 2+2mu -mu)
__device__ __forceinline__ int coarse_nbr(const Geom &g, int a, int d) {
  if (d == 0) return a;
  const int mu = (d - 1) >> 1, dir = (d & 1) ? +1 : -1;
  int bc[4];
  block_coords(g, a, bc);
  int v = bc[mu] + dir;
  if (v < 0) v += g.nb[mu];
  if (v >= g.nb[mu]) v -= g.nb[mu];
  return a + (v - bc[mu]) * g.bstride[mu];
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
template <int NMAX>
__device__ void restrict_block(const Geom &g, int b, const float *V, size_t fstride, int N, const float *in, int face,
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
          load_spinor<float, float>(V + k * fstride, g, b, s, v);
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

template <int NMAX>
__global__ void __launch_bounds__(MG_TPB) k_restrict(Geom g, const float *V, size_t fstride, int N, const float *in,
                                                    float2 *out) {
  restrict_block<NMAX>(g, blockIdx.x, V, fstride, N, in, -1, out + (size_t)blockIdx.x * 2 * N, 1);
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
    restrict_block<NMAX>(g, a, V, fstride, N, w, -1, base + (size_t)col * n2, 1);
  } else if ((diff & (diff - 1)) == 0) {
    const int mu = __ffs(diff) - 1;
    restrict_block<NMAX>(g, a, V, fstride, N, w, 2 * mu + 1, base + ((size_t)(1 + 2 * mu) * n2 + col) * n2, 1);
    restrict_block<NMAX>(g, a, V, fstride, N, w, 2 * mu, base + ((size_t)(2 + 2 * mu) * n2 + col) * n2, 1);
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
__global__ void k_prolong(Geom g, const float *V, size_t fstride, int N, const float2 *c, float *x) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  const float2 *cb = c + (size_t)b * 2 * N;
  float2 o[12];
#pragma unroll
  for (int q = 0; q < 12; q++) o[q] = make_float2(0.f, 0.f);
  for (int k = 0; k < N; k++) {
    Spinor<float> v;
    load_spinor<float, float>(V + k * fstride, g, b, s, v);
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

// y = D_c x: one CTA per aggregate, thread per row (2N <= 64)
__global__ void k_coarse_apply(Geom g, const float2 *__restrict__ Dc, int N, const float2 *__restrict__ x, float2 *y) {
  extern __shared__ float2 xs[];   // [9][2N]
  const int a = blockIdx.x, n2 = 2 * N, row = threadIdx.x;
  for (int q = threadIdx.x; q < 9 * n2; q += blockDim.x) {
    const int d = q / n2, c = q - d * n2;
    xs[q] = x[(size_t)coarse_nbr(g, a, d) * n2 + c];
  }
  __syncthreads();
  if (row >= n2) return;
  float2 acc = make_float2(0.f, 0.f);
  const float2 *D = Dc + (size_t)a * 9 * n2 * n2;
  for (int d = 0; d < 9; d++)
    for (int c = 0; c < n2; c++) acc = cfma(D[((size_t)d * n2 + c) * n2 + row], xs[d * n2 + c], acc);
  y[(size_t)a * n2 + row] = acc;
}

// ---------------------------------------------------------- coarse GMRES
// GMRES(k) on D_c with one cycle of at most `kmax` steps from x = 0 and the
// control (Givens rotations, convergence test) on the device, so a coarse
// solve needs no host synchronisation and can be captured in a CUDA graph.
struct CgState {
  int j, done, steps;
  double bnorm, tol;
  double2 H[65 * 64];
  double2 g[65];
  double cs[64];
  double2 sn[64];
  double2 y[64];
  double hn;
};

constexpr int CG_BLK = 128;   // reduction CTAs for coarse vector norms / updates
constexpr int CG_CHUNKS = 32; // CTAs per coarse dot product

// partial[i][chunk] = this CTA's part of <v_i, w>, i = blockIdx.y < k
__global__ void __launch_bounds__(256) k_cg_dots(const float2 *Vc, size_t n, const float2 *w, double2 *partial,
                                                 const CgState *st) {
  if (st->done) return;
  __shared__ double2 red[8];
  const int i = blockIdx.y;
  double2 acc = make_double2(0, 0);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 we = w[e], v = Vc[i * n + e];
    acc.x += (double)(v.x * we.x + v.y * we.y);
    acc.y += (double)(v.x * we.y - v.y * we.x);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0, 0);
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
      t.x += red[q].x;
      t.y += red[q].y;
    }
    partial[(size_t)i * CG_CHUNKS + blockIdx.x] = t;
  }
}

// H[.., j] = sum of partials (fixed order); k = j + 1 projections
__global__ void k_cg_hcol(const double2 *partial, int k, CgState *st) {
  if (st->done) return;
  const int i = threadIdx.x;
  if (i >= k) return;
  double2 t = make_double2(0, 0);
  for (int b = 0; b < CG_CHUNKS; b++) {
    t.x += partial[(size_t)i * CG_CHUNKS + b].x;
    t.y += partial[(size_t)i * CG_CHUNKS + b].y;
  }
  st->H[i * 64 + st->j] = t;
}

// w -= sum_i H[i][j] v_i ; partial[blk] = |w|^2
__global__ void __launch_bounds__(256) k_cg_axpy(const float2 *Vc, size_t n, int k, float2 *w, double *partial,
                                                 const CgState *st) {
  if (st->done) return;
  __shared__ float2 hs[64];
  __shared__ double red[8];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double2 h = st->H[i * 64 + st->j];
    hs[i] = make_float2((float)h.x, (float)h.y);
  }
  __syncthreads();
  double nrm = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float2 we = w[e];
    for (int i = 0; i < k; i++) {
      const float2 v = Vc[i * n + e], h = hs[i];
      we.x -= h.x * v.x - h.y * v.y;
      we.y -= h.x * v.y + h.y * v.x;
    }
    w[e] = we;
    nrm += (double)(we.x * we.x + we.y * we.y);
  }
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[q];
    partial[blockIdx.x] = t;
  }
}

// one thread: finish step j (Givens, convergence); set hn for the next basis vector
__global__ void k_cg_givens(const double *partial, int nblk, CgState *st, int kmax) {
  if (st->done) return;
  double n2 = 0;
  for (int b = 0; b < nblk; b++) n2 += partial[b];
  const int j = st->j;
  const double hn = sqrt(n2 > 0 ? n2 : 0);
  for (int i = 0; i < j; i++) {
    double2 a = st->H[i * 64 + j], c = st->H[(i + 1) * 64 + j];
    const double cs = st->cs[i];
    const double2 sn = st->sn[i];
    // a' = cs a + sn c ; c' = -conj(sn) a + cs c
    double2 a2 = make_double2(cs * a.x + sn.x * c.x - sn.y * c.y, cs * a.y + sn.x * c.y + sn.y * c.x);
    double2 c2 = make_double2(-(sn.x * a.x + sn.y * a.y) + cs * c.x, -(sn.x * a.y - sn.y * a.x) + cs * c.y);
    st->H[i * 64 + j] = a2;
    st->H[(i + 1) * 64 + j] = c2;
  }
  const double2 a = st->H[j * 64 + j];
  const double aa = sqrt(a.x * a.x + a.y * a.y), rr = sqrt(aa * aa + hn * hn);
  double cs;
  double2 sn;
  if (aa == 0) {
    cs = 0;
    sn = make_double2(1, 0);
  } else {
    cs = aa / rr;
    sn = make_double2(a.x / aa * hn / rr, a.y / aa * hn / rr);
  }
  st->cs[j] = cs;
  st->sn[j] = sn;
  st->H[j * 64 + j] = make_double2(cs * a.x + sn.x * hn, cs * a.y + sn.y * hn);
  const double2 gj = st->g[j];
  st->g[j + 1] = make_double2(-(sn.x * gj.x + sn.y * gj.y), -(sn.x * gj.y - sn.y * gj.x));
  st->g[j] = make_double2(cs * gj.x, cs * gj.y);
  st->hn = hn;
  st->steps = j + 1;
  const double est = sqrt(st->g[j + 1].x * st->g[j + 1].x + st->g[j + 1].y * st->g[j + 1].y);
  if (est <= st->tol * st->bnorm || hn == 0 || j + 1 >= kmax) st->done = 1;
  st->j = j + 1;
}

// v_{j} = w / hn (the new basis vector), skipped once done
__global__ void k_cg_next(float2 *Vc, size_t n, const float2 *w, const CgState *st) {
  if (st->done) return;
  const float inv = (float)(1.0 / st->hn);
  float2 *v = Vc + (size_t)st->j * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 we = w[e];
    v[e] = make_float2(we.x * inv, we.y * inv);
  }
}

// start: bnorm from partial[0..nblk) (|b|^2), v_0 = b / |b|, g = |b| e_1
__global__ void k_cg_start(const double *partial, int nblk, CgState *st, double tol) {
  double n2 = 0;
  for (int b = 0; b < nblk; b++) n2 += partial[b];
  st->bnorm = sqrt(n2 > 0 ? n2 : 0);
  st->tol = tol;
  st->j = 0;
  st->steps = 0;
  st->done = st->bnorm == 0;
  for (int i = 0; i < 65; i++) st->g[i] = make_double2(0, 0);
  st->g[0] = make_double2(st->bnorm, 0);
  st->hn = st->bnorm;
}

__global__ void k_cg_first(float2 *Vc, size_t n, const float2 *b, const CgState *st) {
  const float inv = st->bnorm > 0 ? (float)(1.0 / st->bnorm) : 0.f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 be = b[e];
    Vc[e] = make_float2(be.x * inv, be.y * inv);
  }
}

// |b|^2 partials
__global__ void __launch_bounds__(256) k_cg_norm(const float2 *b, size_t n, double *partial) {
  __shared__ double red[8];
  double nrm = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    nrm += (double)(b[e].x * b[e].x + b[e].y * b[e].y);
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[q];
    partial[blockIdx.x] = t;
  }
}

// back substitution R y = g (one thread)
__global__ void k_cg_solve(CgState *st) {
  const int k = st->steps;
  for (int i = k - 1; i >= 0; i--) {
    double2 t = st->g[i];
    for (int l = i + 1; l < k; l++) {
      const double2 h = st->H[i * 64 + l], yl = st->y[l];
      t.x -= h.x * yl.x - h.y * yl.y;
      t.y -= h.x * yl.y + h.y * yl.x;
    }
    const double2 d = st->H[i * 64 + i];
    const double dd = d.x * d.x + d.y * d.y;
    st->y[i] = dd > 0 ? make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd) : make_double2(0, 0);
  }
}

// x = sum_i y_i v_i
__global__ void k_cg_update(const float2 *Vc, size_t n, float2 *x, const CgState *st) {
  const int k = st->steps;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < k; i++) {
      const double2 y = st->y[i];
      acc = cfma(make_float2((float)y.x, (float)y.y), Vc[i * n + e], acc);
    }
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
  void *p[] = {Vc, w, cb, ce, xf, rf, tf, tin, tout, partial, pnorm, st};
  for (void *q : p)
    if (q) cudaFree(q);
}

int MgWork::init(const Mg *mg) {
  const Geom &g = mg->op->lat->g;
  nc = (size_t)g.nblocks * 2 * mg->N;
  const size_t f32 = (size_t)g.V * 24 * 4, fp = (size_t)g.V * 24 * real_bytes(mg->op->prec);
  const int kmax = mg->p.coarse_max_iter;
  bool ok = cudaMalloc(&Vc, sizeof(float2) * nc * (kmax + 1)) == cudaSuccess &&
            cudaMalloc(&w, sizeof(float2) * nc) == cudaSuccess && cudaMalloc(&cb, sizeof(float2) * nc) == cudaSuccess &&
            cudaMalloc(&ce, sizeof(float2) * nc) == cudaSuccess && cudaMalloc(&xf, f32) == cudaSuccess &&
            cudaMalloc(&rf, f32) == cudaSuccess && cudaMalloc(&tf, f32) == cudaSuccess &&
            cudaMalloc(&tin, fp) == cudaSuccess && cudaMalloc(&tout, fp) == cudaSuccess &&
            cudaMalloc(&partial, sizeof(double2) * CG_CHUNKS * 65) == cudaSuccess &&
            cudaMalloc(&pnorm, sizeof(double) * CG_BLK) == cudaSuccess &&
            cudaMalloc(&st, sizeof(CgState)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    set_error("mg: out of device memory for the coarse-solve workspace");
    return DD_ENOMEM;
  }
  return DD_OK;
}

size_t MgWork::bytes(const Geom &g, int prec, int N, int kmax) {
  const size_t nc = (size_t)g.nblocks * 2 * N;
  return sizeof(float2) * nc * (kmax + 4) + (size_t)g.V * 24 * (4 * 3 + 2 * real_bytes(prec)) +
         sizeof(double2) * CG_CHUNKS * 65 + sizeof(double) * CG_BLK + sizeof(CgState);
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
  if (mg->N <= 8) k_restrict<8><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, mg->N, in, out);
  else if (mg->N <= 16) k_restrict<16><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, mg->N, in, out);
  else k_restrict<32><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, mg->N, in, out);
  return launched("k_restrict");
}

int mg_restrict(const Mg *mg, const float *in, float2 *out, cudaStream_t st) { return restrict_launch(mg, in, out, st); }

int mg_prolong(const Mg *mg, const float2 *c, float *out, cudaStream_t st) {
  const Geom &g = mg->op->lat->g;
  k_prolong<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>(g, mg->V, (size_t)g.V * 24, mg->N, c, out);
  return launched("k_prolong");
}

int mg_coarse_apply(const Mg *mg, const float2 *x, float2 *y, cudaStream_t st) {
  const Geom &g = mg->op->lat->g;
  const int n2 = 2 * mg->N;
  k_coarse_apply<<<g.nblocks, n2 < 32 ? 32 : n2, sizeof(float2) * 9 * n2, st>>>(g, mg->Dc, mg->N, x, y);
  return launched("k_coarse_apply");
}

// e = GMRES_kmax(D_c, b) from 0 (device-side control)
int mg_coarse_solve(const Mg *mg, MgWork &W, const float2 *b, float2 *e, cudaStream_t st) {
  const size_t n = W.nc;
  const int kmax = mg->p.coarse_max_iter;
  CgState *cs = (CgState *)W.st;
  double *pd = W.pnorm;
  k_cg_norm<<<CG_BLK, 256, 0, st>>>(b, n, pd);
  DD_LAUNCHED();
  k_cg_start<<<1, 1, 0, st>>>(pd, CG_BLK, cs, mg->p.coarse_tol);
  DD_LAUNCHED();
  k_cg_first<<<CG_BLK, 256, 0, st>>>(W.Vc, n, b, cs);
  DD_LAUNCHED();
  for (int j = 0; j < kmax; j++) {
    int rc = mg_coarse_apply(mg, W.Vc + (size_t)j * n, W.w, st);
    if (rc) return rc;
    k_cg_dots<<<dim3(CG_CHUNKS, j + 1), 256, 0, st>>>(W.Vc, n, W.w, W.partial, cs);
    DD_LAUNCHED();
    k_cg_hcol<<<1, 64, 0, st>>>(W.partial, j + 1, cs);
    DD_LAUNCHED();
    k_cg_axpy<<<CG_BLK, 256, 0, st>>>(W.Vc, n, j + 1, W.w, pd, cs);
    DD_LAUNCHED();
    k_cg_givens<<<1, 1, 0, st>>>(pd, CG_BLK, cs, kmax);
    DD_LAUNCHED();
    k_cg_next<<<CG_BLK, 256, 0, st>>>(W.Vc, n, W.w, cs);
    DD_LAUNCHED();
  }
  k_cg_solve<<<1, 1, 0, st>>>(cs);
  DD_LAUNCHED();
  k_cg_update<<<CG_BLK, 256, 0, st>>>(W.Vc, n, e, cs);
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
int mg_apply(const Mg *mg, MgWork &W, const float *r, float *x, cudaStream_t st, float scale) {
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

// ------------------------------------------------------------------ setup
static int build_coarse(Mg *mg, cudaStream_t st) {
  const Op *op = mg->op;
  const Geom &g = op->lat->g;
  const size_t fs = (size_t)g.V * 24;
  const int N = mg->N, n2 = 2 * N;
  float *u = nullptr, *wv = nullptr;
  DD_CUDA(cudaMalloc(&u, fs * 4));
  if (cudaMalloc(&wv, fs * 4) != cudaSuccess) {
    cudaFree(u);
    set_error("mg: out of device memory");
    return DD_ENOMEM;
  }
  int rc = cuda_fail(cudaMemsetAsync(mg->Dc, 0, sizeof(float2) * (size_t)g.nblocks * 9 * n2 * n2, st), "memset");
  for (int c16 = 0; c16 < 16 && rc == DD_OK; c16++)
    for (int col = 0; col < n2 && rc == DD_OK; col++) {
      const int hp = col / N, j = col - hp * N;
      k_column<<<(unsigned)((g.V + 127) / 128), 128, 0, st>>>(g, mg->V + j * fs, hp, c16, u);
      if ((rc = launched("k_column"))) break;
      if ((rc = launch_dirac(g, op->f32, u, wv, 1, st))) break;
      if (N <= 8) k_restrict_dc<8><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N, wv, mg->Dc, c16, col);
      else if (N <= 16) k_restrict_dc<16><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N, wv, mg->Dc, c16, col);
      else k_restrict_dc<32><<<g.nblocks, MG_TPB, 0, st>>>(g, mg->V, fs, N, wv, mg->Dc, c16, col);
      rc = launched("k_restrict_dc");
    }
  if (rc == DD_OK) rc = cuda_fail(cudaStreamSynchronize(st), "mg setup");
  cudaFree(u);
  cudaFree(wv);
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
  return build_coarse(mg, st);
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
  Mg *mg = new (std::nothrow) Mg;
  if (!mg) return DD_ENOMEM;
  mg->magic = MAGIC_MG;
  mg->op = op;
  mg->p = *p;
  mg->N = p->n_vectors;
  const size_t n2 = 2 * (size_t)mg->N;
  if (cudaMalloc(&mg->V, (size_t)g.V * 24 * 4 * mg->N) != cudaSuccess ||
      cudaMalloc(&mg->Dc, sizeof(float2) * (size_t)g.nblocks * 9 * n2 * n2) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(mg->V);
    delete mg;
    set_error("dd_create_mg: out of device memory");
    return DD_ENOMEM;
  }
  int rc = mg->work.init(mg);
  if (rc == DD_OK) rc = mg_setup(mg, tv_host, 0);
  if (rc) {
    cudaFree(mg->V);
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
  cudaFree(mg->Dc);
  mg->magic = 0;
  Op *op = mg->op;
  delete mg;
  release_op(op);
}
}  // namespace dd
