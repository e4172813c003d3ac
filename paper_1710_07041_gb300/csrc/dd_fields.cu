// Field set-up kernels: layout conversion (the "data-layout transformation at
// solver entry" of Sec. 5 / Sec. 3.1's adapted layouts), FP16/BF16 storage
// with round-to-nearest-even conversion (Sec. 3.1, Listing 1), and the clover
// term with its even-site inverse.
#include "dd_internal.cuh"

namespace dd {

namespace {

constexpr int TPB = 256;

inline int grid_for(long long n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

// canonical FP64 spinors -> internal layout
template <typename S>
__global__ void k_pack(Geom g, const double2 *__restrict__ canon, void *field, int nrhs, double scale,
                       size_t field_bytes) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V * nrhs) return;
  int r = (int)(t / g.V);
  long long site = t - (long long)r * g.V;
  int b = (int)(site / g.Vb), s = (int)(site - (long long)b * g.Vb);
  long long n = canonical_index(g, b, s);
  const double2 *src = canon + ((long long)r * g.V + n) * 12;
  // narrow directly from the FP64 product so every value is rounded once
  // (round-to-nearest-even for FP16/BF16)
  constexpr int NC = spinor_chunks<S>();
  char *base = (char *)field + r * field_bytes + (size_t)b * g.Vb * spinor_site_bytes(Store<S>::prec) + (size_t)s * 16;
  const size_t cstride = (size_t)g.Vb * 16;
  if constexpr (Store<S>::prec == DD_F16N) {
    // the scale and every component from the FP64 product, each rounded once
    double a[24];
#pragma unroll
    for (int i = 0; i < 12; i++) {
      a[2 * i] = src[i].x * scale;
      a[2 * i + 1] = src[i].y * scale;
    }
    store_fixed16(base, cstride, NC, s, a);
    return;
  }
  using P = typename Store<S>::pair_t;
  constexpr int PPC = Store<S>::reals_per_chunk / 2;  // complex entries per chunk
#pragma unroll
  for (int c = 0; c < NC; c++) {
    uint4 w;
    P *h = (P *)&w;
#pragma unroll
    for (int k = 0; k < PPC; k++) {
      double2 d = src[c * PPC + k];
      h[k] = to_pair<P, double>(d.x * scale, d.y * scale);
    }
    *(uint4 *)(base + c * cstride) = w;
  }
}

template <typename S>
__global__ void k_unpack(Geom g, const void *field, double2 *__restrict__ canon, int nrhs, double scale,
                         size_t field_bytes) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V * nrhs) return;
  int r = (int)(t / g.V);
  long long site = t - (long long)r * g.V;
  int b = (int)(site / g.Vb), s = (int)(site - (long long)b * g.Vb);
  long long n = canonical_index(g, b, s);
  using C = typename Store<S>::comp_t;
  Spinor<C> v;
  load_spinor<S, C>((const char *)field + r * field_bytes, g, b, s, v);
  double2 *dst = canon + ((long long)r * g.V + n) * 12;
#pragma unroll
  for (int i = 0; i < 12; i++) dst[i] = make_double2((double)v.c[i].re * scale, (double)v.c[i].im * scale);
}

template <typename SI, typename SO>
__global__ void k_convert_field(Geom g, const void *in, void *out, int nrhs, double scale, size_t bytes_in,
                                size_t bytes_out) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V * nrhs) return;
  int r = (int)(t / g.V);
  long long site = t - (long long)r * g.V;
  int b = (int)(site / g.Vb), s = (int)(site - (long long)b * g.Vb);
  using C = typename Store<SI>::comp_t;
  using CO = typename Store<SO>::comp_t;
  Spinor<C> v;
  load_spinor<SI, C>((const char *)in + r * bytes_in, g, b, s, v);
  Spinor<CO> w;
#pragma unroll
  for (int i = 0; i < 12; i++) w.c[i] = {(CO)(v.c[i].re * (C)scale), (CO)(v.c[i].im * (C)scale)};
  store_spinor<SO, CO>((char *)out + r * bytes_out, g, b, s, w);
}

// canonical FP64 links [V][4][9] (double2) -> tiles of LP pairs per link:
// LP = 6 (rows 0 and 1; row 2 is rebuilt on load, so the link must be special
// unitary: a deviation of row 2 from conj(row0 x row1) above 1e-6 sets bit 2
// of *bad) or 9 (all entries). CHUNKED: the chunked tile layout (link_slot),
// else pair-major [b][36][Vb].
template <typename P, int LP = link_pairs_of_pair<P>(), bool CHUNKED = true>
__global__ void k_pack_links(Geom g, const double2 *__restrict__ canon, P *out, int *bad) {
  constexpr int CP = chunk_pairs<P>(), NCH = 4 * LP / CP;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  long long n = canonical_index(g, b, s);
  for (int mu = 0; mu < 4; mu++) {
    const double2 *u = canon + n * 36 + 9 * mu;
#pragma unroll
    for (int i = 0; i < LP; i++) {
      const int q = link_slot<CP, LP>(mu, i);
      const size_t at = CHUNKED ? (((size_t)b * NCH + q / CP) * g.Vb + s) * CP + q % CP
                                : ((size_t)b * 4 * LP + LP * mu + i) * g.Vb + s;
      out[at] = to_pair<P, double>(u[i].x, u[i].y);
    }
    if constexpr (LP == 6) {
      double dev = 0;
      for (int k = 0; k < 3; k++) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        // conj(a_k1 b_k2 - a_k2 b_k1), a = row 0, b = row 1
        const double2 a1 = u[k1], a2 = u[k2], b1 = u[3 + k1], b2 = u[3 + k2];
        const double re = (a1.x * b2.x - a1.y * b2.y) - (a2.x * b1.x - a2.y * b1.y);
        const double im = -((a1.x * b2.y + a1.y * b2.x) - (a2.x * b1.y + a2.y * b1.x));
        dev = fmax(dev, fabs(re - u[6 + k].x) + fabs(im - u[6 + k].y));
      }
      if (!(dev <= 1e-6) && bad) atomicOr(bad, 2);
    }
  }
}

// FP64 clover tiles [tile][36][n] (pair-major) -> chunked tiles (clover_slot)
template <typename P>
__global__ void k_convert_clover(const double2 *__restrict__ in, P *out, size_t ntiles, int n) {
  constexpr int CP = chunk_pairs<P>();
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= ntiles * 36 * (size_t)n) return;
  const size_t site = i % n, r = i / n;
  const int pair = (int)(r % 36);
  const size_t tile = r / 36;
  const int q = clover_slot<CP>(pair / 18, pair % 18);
  const double2 d = in[i];
  out[((tile * (36 / CP) + q / CP) * n + site) * CP + q % CP] = to_pair<P, double>(d.x, d.y);
}


// -------------------------------------------------------------- clover
struct M3 { cpx<double> a[9]; };

__device__ inline M3 m3_load(const double2 *canon, long long n, int mu) {
  M3 r;
  const double2 *p = canon + (n * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 9; i++) r.a[i] = {p[i].x, p[i].y};
  return r;
}
__device__ inline M3 m3_mul(const M3 &x, const M3 &y) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cpx<double> s = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) {
        cpx<double> p = cmul(x.a[3 * i + k], y.a[3 * k + j]);
        s.re += p.re;
        s.im += p.im;
      }
      r.a[3 * i + j] = s;
    }
  return r;
}
__device__ inline M3 m3_dag(const M3 &x) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.a[3 * i + j] = {x.a[3 * j + i].re, -x.a[3 * j + i].im};
  return r;
}

struct CanonGeom {
  long long L[4];
};
__device__ inline long long cshift(const CanonGeom &cg, const long long c[4], int mu, int d, int nu, int e) {
  long long x[4] = {c[0], c[1], c[2], c[3]};
  x[mu] = (x[mu] + d + cg.L[mu]) % cg.L[mu];
  if (e) x[nu] = (x[nu] + e + cg.L[nu]) % cg.L[nu];
  return x[0] + cg.L[0] * (x[1] + cg.L[1] * (x[2] + cg.L[2] * x[3]));
}

// F = Q - Q^dagger with Q the sum of the four leaves in the (mu,nu) plane at c
__device__ M3 field_strength(const double2 *U, const CanonGeom &cg, const long long c[4], int mu, int nu) {
  long long n = c[0] + cg.L[0] * (c[1] + cg.L[1] * (c[2] + cg.L[2] * c[3]));
  long long n_pm = cshift(cg, c, mu, 1, nu, 0), n_pn = cshift(cg, c, nu, 1, mu, 0);
  long long n_mm = cshift(cg, c, mu, -1, nu, 0), n_mn = cshift(cg, c, nu, -1, mu, 0);
  long long n_mm_pn = cshift(cg, c, mu, -1, nu, 1), n_mm_mn = cshift(cg, c, mu, -1, nu, -1);
  long long n_mn_pm = cshift(cg, c, nu, -1, mu, 1);
  M3 q, l;
  // n -> n+mu -> n+mu+nu -> n+nu -> n
  q = m3_mul(m3_mul(m3_load(U, n, mu), m3_load(U, n_pm, nu)), m3_mul(m3_dag(m3_load(U, n_pn, mu)), m3_dag(m3_load(U, n, nu))));
  // n -> n+nu -> n+nu-mu -> n-mu -> n
  l = m3_mul(m3_mul(m3_load(U, n, nu), m3_dag(m3_load(U, n_mm_pn, mu))), m3_mul(m3_dag(m3_load(U, n_mm, nu)), m3_load(U, n_mm, mu)));
#pragma unroll
  for (int i = 0; i < 9; i++) { q.a[i].re += l.a[i].re; q.a[i].im += l.a[i].im; }
  // n -> n-mu -> n-mu-nu -> n-nu -> n
  l = m3_mul(m3_mul(m3_dag(m3_load(U, n_mm, mu)), m3_dag(m3_load(U, n_mm_mn, nu))), m3_mul(m3_load(U, n_mm_mn, mu), m3_load(U, n_mn, nu)));
#pragma unroll
  for (int i = 0; i < 9; i++) { q.a[i].re += l.a[i].re; q.a[i].im += l.a[i].im; }
  // n -> n-nu -> n-nu+mu -> n+mu -> n
  l = m3_mul(m3_mul(m3_dag(m3_load(U, n_mn, nu)), m3_load(U, n_mn, mu)), m3_mul(m3_load(U, n_mn_pm, nu), m3_dag(m3_load(U, n, mu))));
#pragma unroll
  for (int i = 0; i < 9; i++) { q.a[i].re += l.a[i].re; q.a[i].im += l.a[i].im; }
  M3 f;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++)
      f.a[3 * i + j] = {q.a[3 * i + j].re - q.a[3 * j + i].re, q.a[3 * i + j].im + q.a[3 * j + i].im};
  return f;
}

// Gauss-Jordan inverse of a 6x6 complex matrix (row-major), partial pivoting.
__device__ bool inv6(cpx<double> *a, cpx<double> *inv) {
  for (int i = 0; i < 36; i++) inv[i] = {(i % 7 == 0) ? 1.0 : 0.0, 0.0};
  for (int c = 0; c < 6; c++) {
    int p = c;
    double best = a[6 * c + c].re * a[6 * c + c].re + a[6 * c + c].im * a[6 * c + c].im;
    for (int r = c + 1; r < 6; r++) {
      double v = a[6 * r + c].re * a[6 * r + c].re + a[6 * r + c].im * a[6 * r + c].im;
      if (v > best) { best = v; p = r; }
    }
    if (!(best > 1e-300)) return false;
    if (p != c)
      for (int j = 0; j < 6; j++) {
        cpx<double> t = a[6 * c + j]; a[6 * c + j] = a[6 * p + j]; a[6 * p + j] = t;
        t = inv[6 * c + j]; inv[6 * c + j] = inv[6 * p + j]; inv[6 * p + j] = t;
      }
    cpx<double> piv = a[6 * c + c];
    cpx<double> ip = {piv.re / best, -piv.im / best};
    for (int j = 0; j < 6; j++) { a[6 * c + j] = cmul(a[6 * c + j], ip); inv[6 * c + j] = cmul(inv[6 * c + j], ip); }
    for (int r = 0; r < 6; r++) {
      if (r == c) continue;
      cpx<double> f = a[6 * r + c];
      for (int j = 0; j < 6; j++) {
        cpx<double> t = cmul(f, a[6 * c + j]);
        a[6 * r + j].re -= t.re; a[6 * r + j].im -= t.im;
        t = cmul(f, inv[6 * c + j]);
        inv[6 * r + j].re -= t.re; inv[6 * r + j].im -= t.im;
      }
    }
  }
  return true;
}

// pack a Hermitian 6x6 (row-major) into 18 pairs; off-diagonals averaged
// from (i,j) and conj(j,i) so the stored block is exactly Hermitian
__device__ inline void pack_herm(const cpx<double> *m, double2 *dst, size_t stride) {
  dst[0] = make_double2(m[0].re, m[7].re);
  dst[stride] = make_double2(m[14].re, m[21].re);
  dst[2 * stride] = make_double2(m[28].re, m[35].re);
  for (int i = 0; i < 6; i++)
    for (int j = i + 1; j < 6; j++) {
      cpx<double> a = m[6 * i + j], b = m[6 * j + i];
      dst[(size_t)herm_off(i, j) * stride] = make_double2(0.5 * (a.re + b.re), 0.5 * (a.im - b.im));
    }
}

__global__ void k_build_clover(Geom g, const double2 *__restrict__ U, double c_sw, double m0, double2 *clov,
                               double2 *cinv, int *bad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  Site st = decode(g, b, s);
  CanonGeom cg;
  long long c[4];
  for (int mu = 0; mu < 4; mu++) {
    cg.L[mu] = g.L[mu];
    c[mu] = (long long)st.bc[mu] * g.bd[mu] + st.lc[mu];
  }
  // planes: xy, xz, yz, xt, yt, zt
  M3 Fxy = field_strength(U, cg, c, 0, 1), Fxz = field_strength(U, cg, c, 0, 2), Fyz = field_strength(U, cg, c, 1, 2);
  M3 Fxt = field_strength(U, cg, c, 0, 3), Fyt = field_strength(U, cg, c, 1, 3), Fzt = field_strength(U, cg, c, 2, 3);
  const double k = -c_sw / 16.0;
  for (int h = 0; h < 2; h++) {
    double sg = h ? 1.0 : -1.0;
    // block = (4 + m0) + k * [[iR, iP + Q], [iP - Q, -iR]]
    cpx<double> M[36];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        int e = 3 * i + j;
        cpx<double> P = {Fyz.a[e].re + sg * Fxt.a[e].re, Fyz.a[e].im + sg * Fxt.a[e].im};
        cpx<double> Q = {-Fxz.a[e].re + sg * Fyt.a[e].re, -Fxz.a[e].im + sg * Fyt.a[e].im};
        cpx<double> R = {Fxy.a[e].re + sg * Fzt.a[e].re, Fxy.a[e].im + sg * Fzt.a[e].im};
        cpx<double> iR = {-R.im, R.re}, iP = {-P.im, P.re};
        M[6 * i + j] = {k * iR.re, k * iR.im};
        M[6 * (i + 3) + (j + 3)] = {-k * iR.re, -k * iR.im};
        M[6 * i + (j + 3)] = {k * (iP.re + Q.re), k * (iP.im + Q.im)};
        M[6 * (i + 3) + j] = {k * (iP.re - Q.re), k * (iP.im - Q.im)};
      }
    for (int i = 0; i < 6; i++) M[7 * i].re += 4.0 + m0;
    pack_herm(M, clov + ((size_t)b * 36 + 18 * h) * g.Vb + s, g.Vb);
    if (st.p == 0) {
      cpx<double> A[36], Ai[36];
      for (int i = 0; i < 36; i++) A[i] = M[i];
      if (!inv6(A, Ai)) atomicOr(bad, 1);
      pack_herm(Ai, cinv + ((size_t)b * 36 + 18 * h) * g.Vh + s, g.Vh);
    }
  }
}

// Caller-supplied site blocks A(n), canonical order [V][2][6][6] complex:
// packed (Hermitian part, as pack_herm) into the tile layout, and the
// even-site blocks inverted.
__global__ void k_load_clover(Geom g, const double2 *__restrict__ A_canon, double2 *clov, double2 *cinv, int *bad) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V) return;
  int b = (int)(t / g.Vb), s = (int)(t - (long long)b * g.Vb);
  const long long n = canonical_index(g, b, s);
  const bool even = s < g.Vh;
  for (int h = 0; h < 2; h++) {
    cpx<double> M[36];
    for (int i = 0; i < 36; i++) {
      const double2 v = A_canon[(n * 2 + h) * 36 + i];
      M[i] = {v.x, v.y};
    }
    pack_herm(M, clov + ((size_t)b * 36 + 18 * h) * g.Vb + s, g.Vb);
    if (even) {
      // invert the stored (exactly Hermitian) block
      cpx<double> A[36], Ai[36];
      for (int i = 0; i < 6; i++) {
        A[7 * i] = {M[7 * i].re, 0.0};
        for (int j = i + 1; j < 6; j++) {
          const cpx<double> a = M[6 * i + j], c = M[6 * j + i];
          A[6 * i + j] = {0.5 * (a.re + c.re), 0.5 * (a.im - c.im)};
          A[6 * j + i] = {A[6 * i + j].re, -A[6 * i + j].im};
        }
      }
      if (!inv6(A, Ai)) atomicOr(bad, 1);
      pack_herm(Ai, cinv + ((size_t)b * 36 + 18 * h) * g.Vh + s, g.Vh);
    }
  }
}

template <typename S> int pack_t(const Geom &g, const double *canon, void *field, int nrhs, double scale, cudaStream_t st) {
  size_t fb = field_bytes(g, Store<S>::prec);
  k_pack<S><<<grid_for(g.V * nrhs), TPB, 0, st>>>(g, (const double2 *)canon, field, nrhs, scale, fb);
  return launched("k_pack");
}
template <typename S> int unpack_t(const Geom &g, const void *field, double *canon, int nrhs, double scale, cudaStream_t st) {
  size_t fb = field_bytes(g, Store<S>::prec);
  k_unpack<S><<<grid_for(g.V * nrhs), TPB, 0, st>>>(g, field, (double2 *)canon, nrhs, scale, fb);
  return launched("k_unpack");
}

template <typename SI, typename SO>
int convert_t(const Geom &g, const void *in, void *out, int nrhs, double scale, cudaStream_t st) {
  k_convert_field<SI, SO><<<grid_for(g.V * nrhs), TPB, 0, st>>>(g, in, out, nrhs, scale, field_bytes(g, Store<SI>::prec),
                                                                field_bytes(g, Store<SO>::prec));
  return launched("k_convert_field");
}

template <typename SI>
int convert_out(const Geom &g, const void *in, int po, void *out, int nrhs, double scale, cudaStream_t st) {
  switch (po) {
    case DD_F64: return convert_t<SI, double>(g, in, out, nrhs, scale, st);
    case DD_F32: return convert_t<SI, float>(g, in, out, nrhs, scale, st);
    case DD_F16: return convert_t<SI, __half>(g, in, out, nrhs, scale, st);
    case DD_BF16: return convert_t<SI, __nv_bfloat16>(g, in, out, nrhs, scale, st);
    case DD_F16N: return convert_t<SI, hn16>(g, in, out, nrhs, scale, st);
  }
  set_error("bad precision %d", po);
  return DD_EINVAL;
}

}  // namespace

int launch_pack(const Geom &g, int prec, const double *canon, void *field, int nrhs, double scale, cudaStream_t st) {
  switch (prec) {
    case DD_F64: return pack_t<double>(g, canon, field, nrhs, scale, st);
    case DD_F32: return pack_t<float>(g, canon, field, nrhs, scale, st);
    case DD_F16: return pack_t<__half>(g, canon, field, nrhs, scale, st);
    case DD_BF16: return pack_t<__nv_bfloat16>(g, canon, field, nrhs, scale, st);
    case DD_F16N: return pack_t<hn16>(g, canon, field, nrhs, scale, st);
  }
  set_error("bad precision %d", prec);
  return DD_EINVAL;
}

int launch_unpack(const Geom &g, int prec, const void *field, double *canon, int nrhs, double scale, cudaStream_t st) {
  switch (prec) {
    case DD_F64: return unpack_t<double>(g, field, canon, nrhs, scale, st);
    case DD_F32: return unpack_t<float>(g, field, canon, nrhs, scale, st);
    case DD_F16: return unpack_t<__half>(g, field, canon, nrhs, scale, st);
    case DD_BF16: return unpack_t<__nv_bfloat16>(g, field, canon, nrhs, scale, st);
    case DD_F16N: return unpack_t<hn16>(g, field, canon, nrhs, scale, st);
  }
  set_error("bad precision %d", prec);
  return DD_EINVAL;
}

int launch_convert_clover(int prec, const double *in, void *out, size_t ntiles, int n, cudaStream_t st) {
  const double2 *c = (const double2 *)in;
  const size_t total = ntiles * 36 * (size_t)n;
  const unsigned grid = (unsigned)((total + TPB - 1) / TPB);
  switch (prec) {
    case DD_F64: k_convert_clover<double2><<<grid, TPB, 0, st>>>(c, (double2 *)out, ntiles, n); break;
    case DD_F32: k_convert_clover<float2><<<grid, TPB, 0, st>>>(c, (float2 *)out, ntiles, n); break;
    case DD_F16:
    case DD_F16N: k_convert_clover<__half2><<<grid, TPB, 0, st>>>(c, (__half2 *)out, ntiles, n); break;
    case DD_BF16: k_convert_clover<__nv_bfloat162><<<grid, TPB, 0, st>>>(c, (__nv_bfloat162 *)out, ntiles, n); break;
    default: set_error("bad precision %d", prec); return DD_EINVAL;
  }
  return launched("k_convert_clover");
}

int launch_convert_field(const Geom &g, int pi, const void *in, int po, void *out, int nrhs, double scale,
                         cudaStream_t st) {
  switch (pi) {
    case DD_F64: return convert_out<double>(g, in, po, out, nrhs, scale, st);
    case DD_F32: return convert_out<float>(g, in, po, out, nrhs, scale, st);
    case DD_F16: return convert_out<__half>(g, in, po, out, nrhs, scale, st);
    case DD_BF16: return convert_out<__nv_bfloat16>(g, in, po, out, nrhs, scale, st);
    case DD_F16N: return convert_out<hn16>(g, in, po, out, nrhs, scale, st);
  }
  set_error("bad precision %d", pi);
  return DD_EINVAL;
}

int launch_pack_links(const Geom &g, int prec, const double *canon, void *out, int *bad, cudaStream_t st) {
  const double2 *c = (const double2 *)canon;
  switch (prec) {
    case DD_F64: k_pack_links<double2><<<grid_for(g.V), TPB, 0, st>>>(g, c, (double2 *)out, bad); break;
    case DD_F32: k_pack_links<float2><<<grid_for(g.V), TPB, 0, st>>>(g, c, (float2 *)out, bad); break;
    case DD_F16:
    case DD_F16N: k_pack_links<__half2><<<grid_for(g.V), TPB, 0, st>>>(g, c, (__half2 *)out, bad); break;
    case DD_BF16:
      k_pack_links<__nv_bfloat162><<<grid_for(g.V), TPB, 0, st>>>(g, c, (__nv_bfloat162 *)out, bad);
      break;
    default: set_error("bad precision %d", prec); return DD_EINVAL;
  }
  return launched("k_pack_links");
}

int launch_pack_links_full(const Geom &g, int prec, const double *canon, void *out, cudaStream_t st) {
  const double2 *c = (const double2 *)canon;
  switch (prec) {
    case DD_F64: k_pack_links<double2, 9, false><<<grid_for(g.V), TPB, 0, st>>>(g, c, (double2 *)out, nullptr); break;
    case DD_F32: k_pack_links<float2, 9, false><<<grid_for(g.V), TPB, 0, st>>>(g, c, (float2 *)out, nullptr); break;
    case DD_F16:
    case DD_F16N: k_pack_links<__half2, 9, false><<<grid_for(g.V), TPB, 0, st>>>(g, c, (__half2 *)out, nullptr); break;
    case DD_BF16:
      k_pack_links<__nv_bfloat162, 9, false><<<grid_for(g.V), TPB, 0, st>>>(g, c, (__nv_bfloat162 *)out, nullptr);
      break;
    default: set_error("bad precision %d", prec); return DD_EINVAL;
  }
  return launched("k_pack_links");
}


// FP64 complex -> double-float: hi = RN(v), lo = RN(v - hi) (v - hi is exact)
__global__ void k_split_pairs(const double2 *__restrict__ in, float4 *out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 d = in[i];
    const float rh = __double2float_rn(d.x), ih = __double2float_rn(d.y);
    out[i] = make_float4(rh, __double2float_rn(d.x - (double)rh), ih, __double2float_rn(d.y - (double)ih));
  }
}

int launch_split_pairs(const double *in, void *out, size_t n, cudaStream_t st) {
  k_split_pairs<<<2048, 256, 0, st>>>((const double2 *)in, (float4 *)out, n);
  return launched("k_split_pairs");
}

int launch_load_clover(const Geom &g, const double *A_canon, double *clov64, double *cinv64, int *bad,
                       cudaStream_t st) {
  k_load_clover<<<grid_for(g.V, 128), 128, 0, st>>>(g, (const double2 *)A_canon, (double2 *)clov64,
                                                   (double2 *)cinv64, bad);
  return launched("k_load_clover");
}

int launch_build_clover(const Geom &g, const double *links_canon, double c_sw, double m0, double *clov64,
                        double *cinv64, int *bad, cudaStream_t st) {
  k_build_clover<<<grid_for(g.V, 128), 128, 0, st>>>(g, (const double2 *)links_canon, c_sw, m0, (double2 *)clov64,
                                                   (double2 *)cinv64, bad);
  return launched("k_build_clover");
}

}  // namespace dd
