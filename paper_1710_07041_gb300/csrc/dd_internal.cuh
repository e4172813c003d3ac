// Internal declarations shared by the library's CUDA translation units.
//
// Layout in HBM. Every field is stored block-major so that one Schwarz block
// (the SAP "domain" of Sec. 3.1) is a contiguous tile:
//   tile index b = lexicographic block coordinate (x fastest),
//   inside a tile: even-parity sites first, then odd; within a parity the
//   position is (local lexicographic index) / 2.
// A spinor field of precision P is [block][chunk][Vb] with 16-byte chunks
// (F64: 2 reals, F32: 4 reals, F16/BF16: 8 reals), so a warp reading one chunk
// of 32 consecutive sites issues one fully coalesced 512-byte request.
// Links and clover site blocks are tiles of "pairs" of two reals (double2 /
// float2 / half2). The Dslash's links: 4 links x 18 reals = 72 reals per site
// in FP64, the first two rows only (48 reals) in 32- and 16-bit storage (see
// link_pairs), in the chunked tile layout (see chunk_pairs); the Schwarz
// kernel's links: all 72 reals, pair-major [block][36][Vb]. Clover: 2
// chirality blocks x 36 reals (6 real diagonal + 15 complex upper entries,
// row-major) = 72 reals per site, chunked tiles of Vb sites; the even-site
// inverse clover, chunked tiles of Vb/2 sites.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <type_traits>

#include "../../include/dd.h"

#include <nvtx3/nvToolsExt.h>

namespace dd {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *where);
// Count a kernel launch and report a launch error (if any).
int launched(const char *where);
void count_launches(int n);  // kernels launched through a replayed graph
#define DD_LAUNCHED()                          \
  do {                                         \
    int rc_ = ::dd::launched("kernel launch"); \
    if (rc_) return rc_;                       \
  } while (0)
#define DD_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::dd::cuda_fail(e_, #call);  \
  } while (0)

// -------------------------------------------------------------- geometry
struct Geom {
  int L[4];         // extents by direction: 0:x 1:y 2:z 3:t
  int bd[4];        // block extents (powers of two >= 2)
  int lbd[4];       // log2 of block extents
  int nb[4];        // blocks per direction
  int bstride[4];   // block-index stride per direction
  int Vb, Vh;       // sites per block, per block and parity
  int nblocks;
  long long V;
  int antiperiodic;
};

// Decoded site: block b, position s in the tile, local and block coordinates.
struct Site {
  int b, s, p;      // block, tile position, parity
  int lc[4];        // local coordinates
  int bc[4];        // block coordinates
};

__host__ __device__ inline int parity_of(const int lc[4]) { return (lc[0] + lc[1] + lc[2] + lc[3]) & 1; }

__host__ __device__ inline int local_lex(const Geom &g, const int lc[4]) {
  return lc[0] + ((lc[1] + ((lc[2] + (lc[3] << g.lbd[2])) << g.lbd[1])) << g.lbd[0]);
}

// tile position s -> local coordinates (inverse of pos_of)
__host__ __device__ inline void local_coords(const Geom &g, int s, int lc[4]) {
  int p = s >= g.Vh;
  int j = s - p * g.Vh;
  int k = 2 * j;
  int x0 = k & (g.bd[0] - 1);
  int r = k >> g.lbd[0];
  lc[1] = r & (g.bd[1] - 1);
  r >>= g.lbd[1];
  lc[2] = r & (g.bd[2] - 1);
  lc[3] = r >> g.lbd[2];
  int q = (lc[1] + lc[2] + lc[3]) & 1;
  lc[0] = x0 + (p ^ q);
}

__host__ __device__ inline int pos_of(const Geom &g, const int lc[4]) {
  return parity_of(lc) * g.Vh + (local_lex(g, lc) >> 1);
}

__host__ __device__ inline void block_coords(const Geom &g, int b, int bc[4]) {
  bc[0] = b % g.nb[0];
  int r = b / g.nb[0];
  bc[1] = r % g.nb[1];
  r /= g.nb[1];
  bc[2] = r % g.nb[2];
  bc[3] = r / g.nb[2];
}

__host__ __device__ inline Site decode(const Geom &g, int b, int s) {
  Site t;
  t.b = b;
  t.s = s;
  t.p = s >= g.Vh;
  local_coords(g, s, t.lc);
  block_coords(g, b, t.bc);
  return t;
}

// Neighbour of site t in direction mu (dir = +1 / -1): its block and tile
// position; *sign is -1 for a hop across the antiperiodic time edge; *inside
// tells whether it lies in the same block.
__host__ __device__ inline void neighbour(const Geom &g, const Site &t, int mu, int dir, int *nb_b,
                                          int *nb_s, float *sign, bool *inside) {
  int lc[4] = {t.lc[0], t.lc[1], t.lc[2], t.lc[3]};
  int v = lc[mu] + dir;
  int b = t.b;
  *sign = 1.f;
  *inside = true;
  if (v < 0 || v >= g.bd[mu]) {
    *inside = false;
    v &= g.bd[mu] - 1;
    int bcv = t.bc[mu] + dir;
    if (bcv < 0) {
      bcv += g.nb[mu];
      if (mu == 3 && g.antiperiodic) *sign = -1.f;
    } else if (bcv >= g.nb[mu]) {
      bcv -= g.nb[mu];
      if (mu == 3 && g.antiperiodic) *sign = -1.f;
    }
    b += (bcv - t.bc[mu]) * g.bstride[mu];
  }
  lc[mu] = v;
  *nb_b = b;
  *nb_s = pos_of(g, lc);
}

// canonical (lexicographic) site index of (b, s)
__host__ __device__ inline long long canonical_index(const Geom &g, int b, int s) {
  Site t = decode(g, b, s);
  long long c[4];
  for (int mu = 0; mu < 4; mu++) c[mu] = (long long)t.bc[mu] * g.bd[mu] + t.lc[mu];
  return c[0] + g.L[0] * (c[1] + (long long)g.L[1] * (c[2] + (long long)g.L[2] * c[3]));
}

// SHAPE: 0 block shape from g at run time; 1 the 4^4 block, 2 the 8x4^3
// block (T x Z x Y x X) as compile-time constants, so that every tile and
// shared-vector stride is an immediate offset instead of index arithmetic.
template <int SHAPE>
__device__ __forceinline__ Geom block_shape(Geom g) {
  if constexpr (SHAPE == 1) {
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      g.bd[mu] = 4;
      g.lbd[mu] = 2;
    }
    g.Vb = 256;
    g.Vh = 128;
  } else if constexpr (SHAPE == 2) {
#pragma unroll
    for (int mu = 0; mu < 3; mu++) {
      g.bd[mu] = 4;
      g.lbd[mu] = 2;
    }
    g.bd[3] = 8;
    g.lbd[3] = 3;
    g.Vb = 512;
    g.Vh = 256;
  }
  return g;
}
// the SHAPE a launch may use for geometry g (0: none matches)
__host__ __device__ inline int shape_of(const Geom &g) {
  if (g.bd[0] == 4 && g.bd[1] == 4 && g.bd[2] == 4 && g.bd[3] == 4) return 1;
  if (g.bd[0] == 4 && g.bd[1] == 4 && g.bd[2] == 4 && g.bd[3] == 8) return 2;
  return 0;
}

// Checked build (compiled with -DDD_CHECKED; the stand-in for a memory
// checker, which is not available on the target machines): the main global
// and shared-memory access paths check their indices; an index out of range
// is counted and replaced by 0, so no access leaves its buffer, and
// dd_device_status reports the count. Normal builds check nothing.
#ifdef DD_CHECKED
static __device__ unsigned dd_bounds_errors = 0;
#define DD_CHECK_INDEX(i, n)                                              \
  do {                                                                    \
    if ((unsigned long long)(i) >= (unsigned long long)(n)) {             \
      atomicAdd(&dd_bounds_errors, 1u);                                   \
      (i) = 0;                                                            \
    }                                                                     \
  } while (0)
int register_bounds_reader(unsigned (*read)());
// this translation unit's counter, read and cleared (registered at load time)
static unsigned dd_read_bounds_errors() {
  unsigned n = 0, z = 0;
  if (cudaMemcpyFromSymbol(&n, dd_bounds_errors, sizeof n) != cudaSuccess) return 0;
  if (n) cudaMemcpyToSymbol(dd_bounds_errors, &z, sizeof z);
  return n;
}
[[maybe_unused]] static const int dd_bounds_registered = register_bounds_reader(&dd_read_bounds_errors);
#else
#define DD_CHECK_INDEX(i, n) \
  do {                       \
  } while (0)
#endif
// total count of all translation units' checked-build counters (0 unless -DDD_CHECKED)
unsigned bounds_errors_all();

// ------------------------------------------------------------- precisions
template <typename S> struct Store;
template <> struct Store<double> {
  static constexpr int prec = DD_F64;
  static constexpr int reals_per_chunk = 2;   // spinor chunk: double2
  using pair_t = double2;                      // link / clover pair
  using comp_t = double;
};
template <> struct Store<float> {
  static constexpr int prec = DD_F32;
  static constexpr int reals_per_chunk = 4;   // float4
  using pair_t = float2;
  using comp_t = float;
};
template <> struct Store<__half> {
  static constexpr int prec = DD_F16;
  static constexpr int reals_per_chunk = 8;   // 8 halves in a uint4
  using pair_t = __half2;
  using comp_t = float;
};
template <> struct Store<__nv_bfloat16> {
  static constexpr int prec = DD_BF16;
  static constexpr int reals_per_chunk = 8;
  using pair_t = __nv_bfloat162;
  using comp_t = float;
};
// DD_F16N: spinors as 16-bit fixed point with a per-site FP32 scale (see
// dd.h), operator tiles as FP16 pairs
struct hn16 {};
template <> struct Store<hn16> {
  static constexpr int prec = DD_F16N;
  static constexpr int reals_per_chunk = 8;   // 8 int16 in a uint4
  using pair_t = __half2;
  using comp_t = float;
};

// Double-float numbers: an unevaluated sum hi + lo of two FP32 values
// (|lo| <= ulp(hi) / 2), about 48 significant bits, from error-free FP32
// transformations (Knuth's TwoSum, Dekker's FastTwoSum, the FMA-exact
// product). GB300 runs FP64 at a small fraction of its FP32 rate; this type
// runs the true residual's Dslash of a mixed-precision solve on the FP32
// pipes. Each operation has a relative error of a few units of 2^-44 of its
// operands (the "sloppy" double-float add and product). The library is not
// built with reassociating fast-math flags, which would break them.
struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ __forceinline__ dfl(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ __forceinline__ dfl(float v) : hi(v), lo(0.f) {}
  __host__ __device__ __forceinline__ dfl(float h, float l, int) : hi(h), lo(l) {}
};
__device__ __forceinline__ dfl df_fast2(float s, float e) {   // |s| >= |e|
  const float h = s + e;
  return dfl(h, e - (h - s), 0);
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);   // TwoSum error of a.hi + b.hi
  e += a.lo + b.lo;
  return df_fast2(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo, 0); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);              // exact error of the product
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_fast2(p, e);
}
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl &operator-=(dfl &a, dfl b) { return a = a - b; }

// Double-float storage (internal only): a complex number as float4
// {re.hi, re.lo, im.hi, im.lo}, the FP64 fields' layout with each double
// split once into hi + lo.
constexpr int DD_PREC_DF = 100;
struct dfs {};
template <> struct Store<dfs> {
  static constexpr int prec = DD_PREC_DF;
  static constexpr int reals_per_chunk = 2;
  using pair_t = float4;
  using comp_t = dfl;
};

constexpr size_t real_bytes_of(int prec) { return (prec == DD_F64 || prec == DD_PREC_DF) ? 8 : prec == DD_F32 ? 4 : 2; }

// Links in 32- and 16-bit storage keep the first two rows of each SU(3)
// matrix (6 complex = 12 reals); the third row is rebuilt on load as
// conj(row0 x row1), which holds for every special unitary matrix (the
// operator constructors check the gauge field for it). FP64 fields and their
// double-float split keep all nine entries. Pairs per link:
template <typename S> __host__ __device__ constexpr int link_pairs() {
  return (Store<S>::prec == DD_F64 || Store<S>::prec == DD_PREC_DF) ? 9 : 6;
}
template <typename P> __host__ __device__ constexpr int link_pairs_of_pair() {
  return (std::is_same<P, double2>::value || std::is_same<P, float4>::value) ? 9 : 6;
}
inline int link_pairs_of(int prec) { return (prec == DD_F64 || prec == DD_PREC_DF) ? 9 : 6; }

// Chunked pair tiles (the Dslash's links, and the clover site blocks of every
// kernel): the pairs of one site are grouped into 16-byte chunks of
// CP = 16 / sizeof(pair) pairs (FP64 and double-float 1, FP32 2, FP16/BF16
// 4), [tile][chunk][tile sites][CP], so that a thread reads its pairs with
// 16-byte loads and a warp's load of one chunk over 32 consecutive sites is
// one contiguous 512-byte request. With CP = 1 this is the pair-major layout
// [tile][pair][tile sites]. A site's pairs take slots 0 .. 4 LP - 1 (links)
// or 0 .. 35 (clover); slot q lies in chunk q / CP at position q % CP.
template <typename P> __host__ __device__ constexpr int chunk_pairs() { return 16 / (int)sizeof(P); }
inline int chunk_pairs_of(int prec) { return 16 / (int)(2 * real_bytes_of(prec)); }
// Slot of entry i of link mu. With CP = 4 and two-row links (6 pairs) the
// first four pairs of link mu fill chunk mu and the last two share chunk
// 4 + mu / 2 with the next link's (so a link is one 16- and one 8-byte
// load); otherwise in order.
template <int CP, int LP> __host__ __device__ constexpr int link_slot(int mu, int i) {
  return (CP == 4 && LP == 6) ? (i < 4 ? 4 * mu + i : 16 + 2 * mu + (i - 4)) : LP * mu + i;
}
// Slot of entry k (0..17) of clover chirality block h. With CP = 4 the first
// sixteen entries of block h fill chunks 4h .. 4h+3 and the last two of both
// blocks share chunk 8, so either block is four 16-byte loads and one 8-byte
// load for a run-time h; otherwise in order.
template <int CP> __host__ __device__ constexpr int clover_slot(int h, int k) {
  return CP == 4 ? (k < 16 ? 16 * h + k : 32 + 2 * h + (k - 16)) : 18 * h + k;
}

inline size_t real_bytes(int prec) { return (prec == DD_F64 || prec == DD_PREC_DF) ? 8 : prec == DD_F32 ? 4 : 2; }
// bytes per site of a spinor field (DD_F16N: 24 int16 and one FP32 scale)
__host__ __device__ constexpr size_t spinor_site_bytes(int prec) {
  return prec == DD_F16N ? 52 : 24 * ((prec == DD_F64 || prec == DD_PREC_DF) ? 8 : prec == DD_F32 ? 4 : 2);
}
inline size_t field_bytes(const Geom &g, int prec) { return (size_t)g.V * spinor_site_bytes(prec); }
// the storage precisions an operator or field may have
inline bool storage_prec(int prec) {
  return prec == DD_F64 || prec == DD_F32 || prec == DD_F16 || prec == DD_BF16 || prec == DD_F16N;
}
// 16-bit operator tiles (a separate smoother copy of the operator)
inline bool half_tiles(int prec) { return prec == DD_F16 || prec == DD_BF16 || prec == DD_F16N; }
inline size_t pair_bytes(int prec) { return 2 * real_bytes(prec); }

template <typename S> __host__ __device__ constexpr int spinor_chunks() { return 24 / Store<S>::reals_per_chunk; }

// pair conversions (round to nearest even on narrowing)
template <typename C> struct cpx { C re, im; };

template <typename C, typename P> __device__ __forceinline__ cpx<C> from_pair(P v);
template <> __device__ __forceinline__ cpx<double> from_pair<double, double2>(double2 v) { return {v.x, v.y}; }
template <> __device__ __forceinline__ cpx<float> from_pair<float, float2>(float2 v) { return {v.x, v.y}; }
template <> __device__ __forceinline__ cpx<float> from_pair<float, __half2>(__half2 v) {
  float2 f = __half22float2(v);
  return {f.x, f.y};
}
template <> __device__ __forceinline__ cpx<float> from_pair<float, __nv_bfloat162>(__nv_bfloat162 v) {
  float2 f = __bfloat1622float2(v);
  return {f.x, f.y};
}

template <> __device__ __forceinline__ cpx<dfl> from_pair<dfl, float4>(float4 v) {
  return {dfl(v.x, v.y, 0), dfl(v.z, v.w, 0)};
}
template <typename P, typename C> __device__ __forceinline__ P to_pair(C re, C im);
template <> __device__ __forceinline__ double2 to_pair<double2, double>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 to_pair<float2, float>(float re, float im) { return make_float2(re, im); }
template <> __device__ __forceinline__ __half2 to_pair<__half2, float>(float re, float im) {
  return __floats2half2_rn(re, im);
}
template <> __device__ __forceinline__ __nv_bfloat162 to_pair<__nv_bfloat162, float>(float re, float im) {
  return __floats2bfloat162_rn(re, im);
}
template <> __device__ __forceinline__ float2 to_pair<float2, double>(double re, double im) {
  return make_float2((float)re, (float)im);
}
template <> __device__ __forceinline__ __half2 to_pair<__half2, double>(double re, double im) {
  return __halves2half2(__double2half(re), __double2half(im));
}
template <> __device__ __forceinline__ __nv_bfloat162 to_pair<__nv_bfloat162, double>(double re, double im) {
  return __halves2bfloat162(__double2bfloat16(re), __double2bfloat16(im));
}

// ---------------------------------------------------------- spinor access
// A spinor in registers: 12 complex, index 3*spin + colour.
template <typename C> struct Spinor { cpx<C> c[12]; };

// a compute value as FP64
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(dfl v) { return (double)v.hi + (double)v.lo; }

// One site of a DD_F16N field from its 24 real components a (FP32): the
// scale n = max |a_i| (FP32), q_i = round-to-nearest-even(a_i 32767 / n),
// |q_i| <= 32767 (n = 0: zeros). base: the site's first chunk; cstride: bytes
// between chunk rows; the scale row follows the NC chunk rows.
template <typename R>
__device__ __forceinline__ void store_fixed16(char *base, size_t cstride, int NC, int s, const R *a) {
  R m = 0;
#pragma unroll
  for (int i = 0; i < 24; i++) m = fmax(m, fabs(a[i]));
  const float n = (float)m;
  const R inv = n > 0.0f ? (R)32767 / (R)n : (R)0;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    uint4 w;
    short *q = (short *)&w;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const R x = a[8 * c + k] * inv;
      q[k] = (short)fmin(fmax(rint(x), (R)-32767), (R)32767);
    }
    *(uint4 *)(base + c * cstride) = w;
  }
  ((float *)(base - (size_t)s * 16 + NC * cstride))[s] = n;
}

// Load spinor (b, s) from a field of storage S.
template <typename S, typename C>
__device__ __forceinline__ void load_spinor(const void *field, const Geom &g, int b, int s, Spinor<C> &out) {
  DD_CHECK_INDEX(b, g.nblocks);
  DD_CHECK_INDEX(s, g.Vb);
  constexpr int NC = spinor_chunks<S>();
  const char *base = (const char *)field + (size_t)b * g.Vb * spinor_site_bytes(Store<S>::prec) + (size_t)s * 16;
  const size_t cstride = (size_t)g.Vb * 16;
  if constexpr (Store<S>::prec == DD_F16N) {
    // the site's scale follows the block's NC chunk rows
    const float n = __ldg((const float *)(base - (size_t)s * 16 + NC * cstride) + s) * (1.0f / 32767.0f);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint4 v = __ldg((const uint4 *)(base + c * cstride));
      const short *q = (const short *)&v;
#pragma unroll
      for (int k = 0; k < 4; k++) out.c[4 * c + k] = {(C)((float)q[2 * k] * n), (C)((float)q[2 * k + 1] * n)};
    }
  } else if constexpr (Store<S>::prec == DD_F64) {
#pragma unroll
    for (int c = 0; c < 12; c++) {
      double2 v = __ldg((const double2 *)(base + c * cstride));
      out.c[c] = {(C)v.x, (C)v.y};
    }
  } else if constexpr (Store<S>::prec == DD_PREC_DF) {
#pragma unroll
    for (int c = 0; c < 12; c++) out.c[c] = from_pair<C, float4>(__ldg((const float4 *)(base + c * cstride)));
  } else if constexpr (Store<S>::prec == DD_F32) {
#pragma unroll
    for (int c = 0; c < 6; c++) {
      float4 v = __ldg((const float4 *)(base + c * cstride));
      out.c[2 * c] = {(C)v.x, (C)v.y};
      out.c[2 * c + 1] = {(C)v.z, (C)v.w};
    }
  } else {
    using P = typename Store<S>::pair_t;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 v = __ldg((const uint4 *)(base + c * cstride));
      const P *h = (const P *)&v;
#pragma unroll
      for (int k = 0; k < 4; k++) out.c[4 * c + k] = from_pair<C, P>(h[k]);
    }
  }
}

template <typename S, typename C>
__device__ __forceinline__ void store_spinor(void *field, const Geom &g, int b, int s, const Spinor<C> &v) {
  DD_CHECK_INDEX(b, g.nblocks);
  DD_CHECK_INDEX(s, g.Vb);
  constexpr int NC = spinor_chunks<S>();
  char *base = (char *)field + (size_t)b * g.Vb * spinor_site_bytes(Store<S>::prec) + (size_t)s * 16;
  const size_t cstride = (size_t)g.Vb * 16;
  if constexpr (Store<S>::prec == DD_F16N) {
    float a[24];
#pragma unroll
    for (int i = 0; i < 12; i++) {
      a[2 * i] = (float)to_d(v.c[i].re);
      a[2 * i + 1] = (float)to_d(v.c[i].im);
    }
    store_fixed16(base, cstride, NC, s, a);
  } else if constexpr (Store<S>::prec == DD_F64) {
#pragma unroll
    for (int c = 0; c < 12; c++) *(double2 *)(base + c * cstride) = make_double2(to_d(v.c[c].re), to_d(v.c[c].im));
  } else if constexpr (Store<S>::prec == DD_F32) {
#pragma unroll
    for (int c = 0; c < 6; c++)
      *(float4 *)(base + c * cstride) =
          make_float4((float)v.c[2 * c].re, (float)v.c[2 * c].im, (float)v.c[2 * c + 1].re, (float)v.c[2 * c + 1].im);
  } else {
    using P = typename Store<S>::pair_t;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 w;
      P *h = (P *)&w;
#pragma unroll
      for (int k = 0; k < 4; k++) h[k] = to_pair<P, C>(v.c[4 * c + k].re, v.c[4 * c + k].im);
      *(uint4 *)(base + c * cstride) = w;
    }
  }
}

// ------------------------------------------------------------ SU(3) hops
template <typename C> struct Link { cpx<C> m[9]; };

template <typename C> __device__ __forceinline__ cpx<C> cmul(cpx<C> a, cpx<C> b);

// Third row of an SU(3) matrix from the first two: conj(row0 x row1).
template <typename C> __device__ __forceinline__ void su3_third_row(Link<C> &u) {
  const cpx<C> *a = u.m, *b = u.m + 3;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
    const cpx<C> p = cmul(a[k1], b[k2]), q = cmul(a[k2], b[k1]);
    u.m[6 + k] = {p.re - q.re, q.im - p.im};
  }
}

// Link U_mu of site (b, s) from a field of storage S with LP pairs per link:
// the Dslash fields (LP = link_pairs<S>(), CHUNKED: the chunked tile layout
// with link_slot), or the Schwarz kernel's (LP = 9, pair-major
// [block][36][Vb], see OpFields::links_full).
template <typename S, typename C, int LP = link_pairs<S>(), bool CHUNKED = true>
__device__ __forceinline__ void load_link(const void *links, const Geom &g, int b, int s, int mu, Link<C> &u) {
  using P = typename Store<S>::pair_t;
  constexpr int CP = chunk_pairs<P>();
  DD_CHECK_INDEX(b, g.nblocks);
  DD_CHECK_INDEX(s, g.Vb);
  DD_CHECK_INDEX(mu, 4);
  if constexpr (CHUNKED) {
    const uint4 *q = (const uint4 *)links + (size_t)b * (4 * LP / CP) * g.Vb + s;   // chunk c at q[c * Vb]
    if constexpr (CP == 4 && LP == 6) {
      const uint4 v = __ldg(q + (size_t)mu * g.Vb);
      const uint2 w = __ldg((const uint2 *)(q + (size_t)(4 + (mu >> 1)) * g.Vb) + (mu & 1));
      const P *pv = (const P *)&v, *pw = (const P *)&w;
#pragma unroll
      for (int i = 0; i < 4; i++) u.m[i] = from_pair<C, P>(pv[i]);
      u.m[4] = from_pair<C, P>(pw[0]);
      u.m[5] = from_pair<C, P>(pw[1]);
    } else {
      static_assert(LP % CP == 0, "whole chunks per link");
#pragma unroll
      for (int c = 0; c < LP / CP; c++) {
        const uint4 v = __ldg(q + (size_t)(mu * (LP / CP) + c) * g.Vb);
        const P *pv = (const P *)&v;
#pragma unroll
        for (int k = 0; k < CP; k++) u.m[c * CP + k] = from_pair<C, P>(pv[k]);
      }
    }
  } else {
    const P *base = (const P *)links + ((size_t)b * 4 * LP + LP * mu) * g.Vb + s;
#pragma unroll
    for (int i = 0; i < LP; i++) u.m[i] = from_pair<C, P>(__ldg(base + (size_t)i * g.Vb));
  }
  if constexpr (LP == 6) su3_third_row(u);
}

template <typename C> __device__ __forceinline__ cpx<C> cmul(cpx<C> a, cpx<C> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename C> __device__ __forceinline__ cpx<C> cmulc(cpx<C> a, cpx<C> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// c + a b for double-float numbers, accumulated lazily: the product's high
// part is added to c.hi with an error-free TwoSum, its exact rounding error
// (one FMA), the cross terms a.hi b.lo + a.lo b.hi and the sum's error go into
// the low word, which is not renormalised (every consumer reads hi + lo as a
// whole). About 13 FP32 operations instead of a full double-float product
// and sum (~18); the error stays a few units of 2^-44 of the terms.
__device__ __forceinline__ dfl df_mad(dfl a, dfl b, dfl c) {
  const float p = a.hi * b.hi;
  const float pe = fmaf(a.hi, b.hi, -p);
  const float cross = fmaf(a.hi, b.lo, a.lo * b.hi);
  const float s = c.hi + p;
  const float z = s - c.hi;
  const float e = (c.hi - (s - z)) + (p - z);
  return dfl(s, c.lo + (e + (pe + cross)), 0);
}
// Fused multiply-add of the real type: fma for float and double (one
// rounding per term); df_mad for double-float numbers.
template <typename C> __device__ __forceinline__ C mad(C a, C b, C c) {
  if constexpr (std::is_same<C, dfl>::value) return df_mad(a, b, c);
  else return fma(a, b, c);
}
// acc += a b and acc += conj(a) b (complex), as chains of fused multiply-adds
template <typename C> __device__ __forceinline__ void cmac(cpx<C> &acc, cpx<C> a, cpx<C> b) {
  acc.re = mad(a.re, b.re, acc.re);
  acc.re = mad(-a.im, b.im, acc.re);
  acc.im = mad(a.re, b.im, acc.im);
  acc.im = mad(a.im, b.re, acc.im);
}
template <typename C> __device__ __forceinline__ void cmacc(cpx<C> &acc, cpx<C> a, cpx<C> b) {
  acc.re = mad(a.re, b.re, acc.re);
  acc.re = mad(a.im, b.im, acc.re);
  acc.im = mad(a.re, b.im, acc.im);
  acc.im = mad(-a.im, b.re, acc.im);
}

// h = U chi (two spin components of colour vectors)
template <typename C>
__device__ __forceinline__ void su3_mul(const Link<C> &u, const cpx<C> *chi, cpx<C> *h) {
#pragma unroll
  for (int sp = 0; sp < 2; sp++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      cpx<C> a = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) cmac(a, u.m[3 * r + k], chi[3 * sp + k]);
      h[3 * sp + r] = a;
    }
}
// h = U^dagger chi
template <typename C>
__device__ __forceinline__ void su3_dmul(const Link<C> &u, const cpx<C> *chi, cpx<C> *h) {
#pragma unroll
  for (int sp = 0; sp < 2; sp++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      cpx<C> a = {0, 0};
#pragma unroll
      for (int k = 0; k < 3; k++) cmacc(a, u.m[3 * k + r], chi[3 * sp + k]);
      h[3 * sp + r] = a;
    }
}

// Spin projection for a hop in direction MU, chiral basis. FWD: the term
// (1 - g_mu) U_mu(n) psi(n+mu); otherwise (1 + g_mu) U_mu(n-mu)^+ psi(n-mu).
// With g_mu = [[0, A],[A^+, 0]] (A_x = -i s1, A_y = -i s2, A_z = -i s3, A_t = 1):
//   (1 -+ g) psi = [chi ; -+ A^+ chi],  chi = psi_up -+ A psi_down,
// so only the 2-spin chi is multiplied by the link.
template <int MU, bool FWD, typename C>
__device__ __forceinline__ void project(const Spinor<C> &p, cpx<C> *chi) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    cpx<C> u0 = p.c[c], u1 = p.c[3 + c], d0 = p.c[6 + c], d1 = p.c[9 + c];
    if constexpr (MU == 0) {       // A d = (-i d1, -i d0)
      if (FWD) { chi[c] = {u0.re - d1.im, u0.im + d1.re}; chi[3 + c] = {u1.re - d0.im, u1.im + d0.re}; }
      else     { chi[c] = {u0.re + d1.im, u0.im - d1.re}; chi[3 + c] = {u1.re + d0.im, u1.im - d0.re}; }
    } else if constexpr (MU == 1) { // A d = (-d1, d0)
      if (FWD) { chi[c] = {u0.re + d1.re, u0.im + d1.im}; chi[3 + c] = {u1.re - d0.re, u1.im - d0.im}; }
      else     { chi[c] = {u0.re - d1.re, u0.im - d1.im}; chi[3 + c] = {u1.re + d0.re, u1.im + d0.im}; }
    } else if constexpr (MU == 2) { // A d = (-i d0, i d1)
      if (FWD) { chi[c] = {u0.re - d0.im, u0.im + d0.re}; chi[3 + c] = {u1.re + d1.im, u1.im - d1.re}; }
      else     { chi[c] = {u0.re + d0.im, u0.im - d0.re}; chi[3 + c] = {u1.re - d1.im, u1.im + d1.re}; }
    } else {                        // A d = d
      if (FWD) { chi[c] = {u0.re - d0.re, u0.im - d0.im}; chi[3 + c] = {u1.re - d1.re, u1.im - d1.im}; }
      else     { chi[c] = {u0.re + d0.re, u0.im + d0.im}; chi[3 + c] = {u1.re + d1.re, u1.im + d1.im}; }
    }
  }
}

// acc += sgn * reconstruct(h): upper spins h, lower spins -+ A^+ h. With SW
// the two spin halves of acc are stored swapped (upper in c[6..11]).
template <int MU, bool FWD, typename C, bool SW = false>
__device__ __forceinline__ void accum_recon(Spinor<C> &acc, const cpx<C> *h, C sgn) {
  constexpr int UP = SW ? 6 : 0, LO = SW ? 0 : 6;
  // lower spins: acc -= sgn A^+ h (FWD) or += (the entries of A^+ h are
  // entries of h up to sign, so every update is one fused multiply-add)
  const C s = FWD ? -sgn : sgn;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<C> h0 = h[c], h1 = h[3 + c];
    cpx<C> &u0 = acc.c[UP + c], &u1 = acc.c[UP + 3 + c], &l0 = acc.c[LO + c], &l1 = acc.c[LO + 3 + c];
    u0.re = mad(sgn, h0.re, u0.re); u0.im = mad(sgn, h0.im, u0.im);
    u1.re = mad(sgn, h1.re, u1.re); u1.im = mad(sgn, h1.im, u1.im);
    if constexpr (MU == 0) {        // A^+ h = (i h1, i h0)
      l0.re = mad(-s, h1.im, l0.re); l0.im = mad(s, h1.re, l0.im);
      l1.re = mad(-s, h0.im, l1.re); l1.im = mad(s, h0.re, l1.im);
    } else if constexpr (MU == 1) { // A^+ h = (h1, -h0)
      l0.re = mad(s, h1.re, l0.re); l0.im = mad(s, h1.im, l0.im);
      l1.re = mad(-s, h0.re, l1.re); l1.im = mad(-s, h0.im, l1.im);
    } else if constexpr (MU == 2) { // A^+ h = (i h0, -i h1)
      l0.re = mad(-s, h0.im, l0.re); l0.im = mad(s, h0.re, l0.im);
      l1.re = mad(s, h1.im, l1.re); l1.im = mad(-s, h1.re, l1.im);
    } else {                        // A^+ h = h
      l0.re = mad(s, h0.re, l0.re); l0.im = mad(s, h0.im, l0.im);
      l1.re = mad(s, h1.re, l1.re); l1.im = mad(s, h1.im, l1.im);
    }
  }
}

// One hop: acc += sgn * (1 -+ g_mu) W psi, W = U (FWD) or U^dagger (SW: acc's
// spin halves stored swapped).
template <int MU, bool FWD, typename C, bool SW = false>
__device__ __forceinline__ void hop(Spinor<C> &acc, const Link<C> &u, const Spinor<C> &psi, C sgn) {
  cpx<C> chi[6], h[6];
  project<MU, FWD>(psi, chi);
  if (FWD) su3_mul(u, chi, h);
  else su3_dmul(u, chi, h);
  accum_recon<MU, FWD, C, SW>(acc, h, sgn);
}

// ------------------------------------------------------------ clover blocks
// Packed Hermitian 6x6: [0..5] real diagonal as 3 pairs, then 15 complex
// upper entries (i<j) row-major. Pair index of (i,j), i<j:
__host__ __device__ constexpr int herm_off(int i, int j) {
  // entries before row i: sum_{r<i} (5 - r)
  return 3 + (i * (11 - i)) / 2 + (j - i - 1);
}

// y = M x for one packed block (M given as 18 pairs).
template <typename C>
__device__ __forceinline__ void herm6_mv(const cpx<C> *m, const cpx<C> *x, cpx<C> *y) {
  C d[6] = {m[0].re, m[0].im, m[1].re, m[1].im, m[2].re, m[2].im};
#pragma unroll
  for (int i = 0; i < 6; i++) y[i] = {d[i] * x[i].re, d[i] * x[i].im};
#pragma unroll
  for (int i = 0; i < 6; i++)
#pragma unroll
    for (int j = i + 1; j < 6; j++) {
      const cpx<C> a = m[herm_off(i, j)];
      cmac(y[i], a, x[j]);    // y_i += a x_j
      cmacc(y[j], a, x[i]);   // y_j += conj(a) x_i
    }
}

// Chirality block h (18 pairs) of site s from a chunked clover tile whose
// first pair is at tile (n sites per tile; see clover_slot); h may be a
// run-time value. LDG: read through the read-only path (global memory only).
template <bool LDG, typename C, typename P>
__device__ __forceinline__ void clover_block_chunked(const P *tile, size_t n, int s, int h, cpx<C> *m) {
  constexpr int CP = chunk_pairs<P>();
  DD_CHECK_INDEX(s, n);
  DD_CHECK_INDEX(h, 2);
  const uint4 *q = (const uint4 *)tile + s;   // chunk c of site s at q[c * n]
  auto ld4 = [](const uint4 *a) { if constexpr (LDG) return __ldg(a); else return *a; };
  auto ld2 = [](const uint2 *a) { if constexpr (LDG) return __ldg(a); else return *a; };
  if constexpr (CP == 4) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const uint4 v = ld4(q + (size_t)(4 * h + c) * n);
      const P *pv = (const P *)&v;
#pragma unroll
      for (int k = 0; k < 4; k++) m[4 * c + k] = from_pair<C, P>(pv[k]);
    }
    const uint2 w = ld2((const uint2 *)(q + (size_t)8 * n) + h);
    const P *pw = (const P *)&w;
    m[16] = from_pair<C, P>(pw[0]);
    m[17] = from_pair<C, P>(pw[1]);
  } else {
#pragma unroll
    for (int c = 0; c < 18 / CP; c++) {
      const uint4 v = ld4(q + (size_t)((18 / CP) * h + c) * n);
      const P *pv = (const P *)&v;
#pragma unroll
      for (int k = 0; k < CP; k++) m[CP * c + k] = from_pair<C, P>(pv[k]);
    }
  }
}

template <typename S, typename C>
__device__ __forceinline__ void load_clover_block(const void *clov, size_t tile_sites, int b, int s, int h,
                                                  cpx<C> *m) {
  using P = typename Store<S>::pair_t;
  clover_block_chunked<true, C, P>((const P *)clov + (size_t)b * 36 * tile_sites, tile_sites, s, h, m);
}

// out = A psi for a full site (both chirality blocks)
template <typename S, typename C>
__device__ __forceinline__ void clover_apply(const void *clov, size_t tile_sites, int b, int s, const Spinor<C> &in,
                                             Spinor<C> &out) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    cpx<C> m[18];
    load_clover_block<S, C>(clov, tile_sites, b, s, h, m);
    herm6_mv(m, &in.c[6 * h], &out.c[6 * h]);
  }
}

// -------------------------------------------------------------- objects
struct Lattice {
  int magic;
  Geom g;
  int dims[4];
  int block[4];
  int refs;
};

struct Gauge {
  int magic;
  Lattice *lat;
  double *links_canon;   // device [V][4][3][3][2] FP64, canonical order
  int refs;
};

// Operator fields in one storage precision.
struct OpFields {
  int prec = -1;
  void *links = nullptr;  // [nblocks][4 * link_pairs_of(prec)][Vb] pairs (Dslash)
  // [nblocks][36][Vb] pairs, every entry: the Schwarz kernel rebuilds no rows
  // (its block solve reads each link about ten times per phase from L1 or
  // shared memory, where the rebuild would cost more issue slots than the
  // bytes it saves); the same array as `links` for FP64
  void *links_full = nullptr;
  void *clov = nullptr;   // A, chunked tiles of 36 pairs x Vb sites per block (clover_slot)
  void *cinv = nullptr;   // A^-1 on even sites, chunked tiles of 36 pairs x Vh sites
};

struct Op {
  int magic;
  Gauge *gauge;
  Lattice *lat;
  double c_sw, m0;
  int prec;             // smoother precision
  OpFields f64, f32, fp;  // fp = smoother precision fields (aliases f64/f32 when equal)
  OpFields fdf;           // links and A split into double-float (mixed-precision ops: true residual)
  int refs;             // the caller's handle plus multigrid objects built on it
};
void release_op(Op *op);

const OpFields *fields_for(const Op *op, int prec);

// NVTX range for profilers (nsys/ncu --nvtx); costs nothing without a tool
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Per-right-hand-side field pointers, passed to kernels by value so that a
// batch may mix vectors held anywhere in device memory.
constexpr int MAX_RHS = 64;
struct RhsPtrs {
  const void *in[MAX_RHS];
  void *out[MAX_RHS];
  int n = 0;
};
// pointers of nrhs contiguous fields starting at in / out
RhsPtrs contiguous(const void *in, void *out, int nrhs, size_t field_bytes);

// Per-right-hand-side work fields of the Schwarz smoother's incremental
// colour residual (fields of the smoother's storage precision): e[r] the
// latest block corrections, as the face flux into the neighbouring blocks
// (6 complex per face site, see the Schwarz kernel) or, where that does not
// fit a spinor field or for FP64, as a spinor field; r[r] each block's
// residual after its own latest solve (odd sites; the even-site residual of
// an even-odd block solve is zero).
struct AuxPtrs {
  void *e[MAX_RHS];
  void *r[MAX_RHS];
};

// --------------------------------------------------------- kernel launchers
int launch_pack(const Geom &g, int prec, const double *canon, void *field, int nrhs, double scale, cudaStream_t st);
int launch_unpack(const Geom &g, int prec, const void *field, double *canon, int nrhs, double scale, cudaStream_t st);
// FP64 canonical links -> tile layout of `prec`; for 12-real storage raises
// bit 2 of *bad (may be null) if a link is not special unitary to 1e-6
int launch_pack_links(const Geom &g, int prec, const double *links_canon, void *out, int *bad, cudaStream_t st);
// FP64 canonical links -> the full nine-pair tile layout of `prec`
int launch_pack_links_full(const Geom &g, int prec, const double *links_canon, void *out, cudaStream_t st);
// caller-supplied site blocks A(n) [V][2][6][6] complex (canonical order), packed and inverted like the build
int launch_load_clover(const Geom &g, const double *A_canon, double *clov64, double *cinv64, int *bad,
                       cudaStream_t st);
int launch_build_clover(const Geom &g, const double *links_canon, double c_sw, double m0, double *clov64,
                        double *cinv64, int *bad, cudaStream_t st);
// FP64 clover tiles ([tile][36][n] pairs) -> chunked tiles of `prec`
int launch_convert_clover(int prec, const double *in, void *out, size_t ntiles, int n, cudaStream_t st);
int launch_dirac(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st);
int launch_dirac(const Geom &g, const OpFields &f, const void *in, void *out, int nrhs, cudaStream_t st);
// y = D x with double-float fields (f = op->fdf) and double-float inputs p.in
// (FP64 fields split by launch_split_pairs), FP64 outputs p.out
int launch_dirac_df(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st);
// n complex FP64 values -> double-float {hi, lo} pairs, same positions
int launch_split_pairs(const double *in, void *out, size_t n, cudaStream_t st);
// Schwarz sweeps; p.in = right-hand sides b, p.out = iterates x
// One launch of the Schwarz kernel may cover the right-hand sides of several
// lattices (operators) that share the block shape and storage precision:
// group k is a lattice with its operator's fields and the right-hand sides
// rhs0 .. rhs0 + nrhs - 1 of the launch's pointer arrays; its work items are
// item0 .. item0 + (blocks / 2) x ceil(nrhs / tile) - 1.
constexpr int MAX_SAP_GROUPS = 8;
struct SapGroup {
  Geom g;
  const void *links, *clov, *cinv;
  int rhs0, nrhs, item0;
};
struct SapGroups {
  SapGroup grp[MAX_SAP_GROUPS];
  int n, nitems;
};
// A lattice of a multi-lattice smoother launch: geometry, operator fields of
// the smoother precision, and its number of right-hand sides (consecutive in
// the launch's pointer arrays, in the order of the lattices).
struct SapLattice {
  Geom g;
  OpFields f;
  int nrhs;
};
int launch_sap_lattices(const SapLattice *lats, int nlat, const dd_sap_params &sp, const RhsPtrs &p,
                        cudaStream_t st, const AuxPtrs *aux);

// aux (may be null): work fields for the incremental colour residual, one
// pair per right-hand side of p; without them every phase recomputes
// r = b - D x from x
int launch_sap(const Geom &g, const OpFields &f, const dd_sap_params &sp, const RhsPtrs &p, cudaStream_t st,
               const AuxPtrs *aux = nullptr);
// nrhs contiguous fields b, x; aux_base (may be null): 2 x nrhs contiguous
// work fields (e of every right-hand side, then r)
int launch_sap(const Geom &g, const OpFields &f, const dd_sap_params &sp, const void *b, void *x, int nrhs,
               cudaStream_t st, void *aux_base = nullptr);
// DD_OK, or DD_ETIMEOUT if a bounded device wait has expired since the last
// call (waits for the device first; clears the count)
int device_wait_status();
// staging-handshake self-test (see dd_selftest_wait)
int wait_selftest(int expire);
// spinor precision conversion between two internal layouts, y = scale * x
int launch_convert_field(const Geom &g, int prec_in, const void *in, int prec_out, void *out, int nrhs, double scale,
                         cudaStream_t st);

}  // namespace dd
