// Wilson-clover operator y = D x over the whole lattice (Sec. 1's "discretized
// form of the Dirac equation"; the operator every step of the Schwarz method
// of Sec. 3.1 applies):
//   (D x)(n) = A(n) x(n) - 1/2 sum_mu [(1 - g_mu) U_mu(n) x(n+mu) + (1 + g_mu) U_mu(n-mu)^+ x(n-mu)]
// One thread per (site, right-hand side), right-hand side fastest so that the
// threads of one site share its link and clover loads in L1. The kernel is
// HBM-bound: per site it moves 24 (in) + 24 (out) + 72 (links) + 72 (clover)
// reals once, neighbour spinors being re-read from L1/L2.
#include "dd_tune.cuh"

namespace dd {
namespace {

// Like load_spinor, but a DD_F16N site comes back unscaled (its 16-bit
// integers as C): the spinor is out times the returned factor, which the
// caller folds into a later coefficient (one multiply instead of 24). The
// other storages return their values and the factor 1.
template <typename S, typename C>
__device__ __forceinline__ C load_spinor_unscaled(const void *field, const Geom &g, int b, int s, Spinor<C> &out) {
  if constexpr (Store<S>::prec == DD_F16N) {
    DD_CHECK_INDEX(b, g.nblocks);
    DD_CHECK_INDEX(s, g.Vb);
    constexpr int NC = spinor_chunks<S>();
    const char *blk = (const char *)field + (size_t)b * g.Vb * spinor_site_bytes(DD_F16N);
    const size_t cstride = (size_t)g.Vb * 16;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      const uint4 v = __ldg((const uint4 *)(blk + c * cstride + (size_t)s * 16));
      const short *q = (const short *)&v;
#pragma unroll
      for (int k = 0; k < 4; k++) out.c[4 * c + k] = {(C)q[2 * k], (C)q[2 * k + 1]};
    }
    // the site's scale row follows the block's NC chunk rows
    return (C)(__ldg((const float *)(blk + NC * cstride) + s) * (1.0f / 32767.0f));
  } else {
    load_spinor<S, C>(field, g, b, s, out);
    return (C)1;
  }
}

// Loads that bypass L1 (the read-only path without allocating a line): for
// the clover tiles, which the Dslash reads once per site, so that L1 keeps
// the spinor and link lines that neighbouring sites read again.
__device__ __forceinline__ uint4 ld_no_l1(const uint4 *p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_no_l1(const uint2 *p) {
  uint2 v;
  asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

// out = A psi for a full site, as clover_apply, with the tile chunks read by
// ld_no_l1 (the chunked layout of clover_block_chunked: chunk c of site s at
// q[c * n]; with 4 pairs per chunk the last two pairs of both chirality
// blocks share chunk 8)
template <typename S, typename C>
__device__ __forceinline__ void clover_apply_no_l1(const void *clov, size_t n, int b, int s, const Spinor<C> &in,
                                                   Spinor<C> &out) {
  using P = typename Store<S>::pair_t;
  constexpr int CP = chunk_pairs<P>();
  DD_CHECK_INDEX(s, n);
  const uint4 *q = (const uint4 *)((const P *)clov + (size_t)b * 36 * n) + s;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    cpx<C> m[18];
    if constexpr (CP == 4) {
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const uint4 v = ld_no_l1(q + (size_t)(4 * h + c) * n);
        const P *pv = (const P *)&v;
#pragma unroll
        for (int k = 0; k < 4; k++) m[4 * c + k] = from_pair<C, P>(pv[k]);
      }
      const uint2 w = ld_no_l1((const uint2 *)(q + (size_t)8 * n) + h);
      const P *pw = (const P *)&w;
      m[16] = from_pair<C, P>(pw[0]);
      m[17] = from_pair<C, P>(pw[1]);
    } else {
#pragma unroll
      for (int c = 0; c < 18 / CP; c++) {
        const uint4 v = ld_no_l1(q + (size_t)((18 / CP) * h + c) * n);
        const P *pv = (const P *)&v;
#pragma unroll
        for (int k = 0; k < CP; k++) m[CP * c + k] = from_pair<C, P>(pv[k]);
      }
    }
    herm6_mv(m, &in.c[6 * h], &out.c[6 * h]);
  }
}

template <int MU, typename S, typename C>
__device__ __forceinline__ void dirac_dir(const Geom &g, const Site &t, const void *links, const void *in,
                                          Spinor<C> &acc) {
  int nb, ns;
  float sg;
  bool inside;
  Link<C> u;
  Spinor<C> psi;
  // hop coefficient -1/2 (times the antiperiodic sign; for DD_F16N also the
  // neighbour's site scale, its spinor being loaded unscaled)
  auto coef = [&](C f) {
    if constexpr (Store<S>::prec == DD_F16N) return (C)(-0.5f * sg) * f;
    else return (C)(-0.5f * sg);
  };
  neighbour(g, t, MU, +1, &nb, &ns, &sg, &inside);
  C f = load_spinor_unscaled<S, C>(in, g, nb, ns, psi);
  load_link<S, C>(links, g, t.b, t.s, MU, u);
  hop<MU, true>(acc, u, psi, coef(f));
  neighbour(g, t, MU, -1, &nb, &ns, &sg, &inside);
  f = load_spinor_unscaled<S, C>(in, g, nb, ns, psi);
  load_link<S, C>(links, g, nb, ns, MU, u);
  hop<MU, false>(acc, u, psi, coef(f));
}

// TPB threads per CTA; MINB resident CTAs per SM requested from the compiler
// (caps registers so more warps keep loads in flight).
// SHAPE: the block shape as compile-time constants (see block_shape), or 0.
// SO: storage of the output fields (the input's, or FP64 for double-float inputs).
// NL1: the clover tiles read without allocating L1 lines.
template <typename S, int TPB, int MINB, int SHAPE, bool NL1, typename SO = S>
__global__ void __launch_bounds__(TPB, MINB) k_dirac(Geom g_in, const void *__restrict__ links,
                                                     const void *__restrict__ clov, const RhsPtrs p) {
  using C = typename Store<S>::comp_t;
  const Geom g = block_shape<SHAPE>(g_in);
  const int nrhs = p.n;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.V * nrhs) return;
  long long site = t / nrhs;
  int r = (int)(t - site * nrhs);
  int b = (int)(site / g.Vb), s = (int)(site - (long long)b * g.Vb);
  const void *inr = p.in[r];
  Site st = decode(g, b, s);
  Spinor<C> x, acc;
  load_spinor<S, C>(inr, g, b, s, x);
  if constexpr (NL1) clover_apply_no_l1<S, C>(clov, g.Vb, b, s, x, acc);
  else clover_apply<S, C>(clov, g.Vb, b, s, x, acc);
  dirac_dir<0, S, C>(g, st, links, inr, acc);
  dirac_dir<1, S, C>(g, st, links, inr, acc);
  dirac_dir<2, S, C>(g, st, links, inr, acc);
  dirac_dir<3, S, C>(g, st, links, inr, acc);
  store_spinor<SO, C>(p.out[r], g, b, s, acc);
}

template <typename S, int TPB, int MINB, bool NL1, typename SO = S>
int dirac_v(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st) {
  long long n = g.V * p.n;
  const unsigned grid = (unsigned)((n + TPB - 1) / TPB);
  if (shape_of(g) == 1) k_dirac<S, TPB, MINB, 1, NL1, SO><<<grid, TPB, 0, st>>>(g, f.links, f.clov, p);
  else k_dirac<S, TPB, MINB, 0, NL1, SO><<<grid, TPB, 0, st>>>(g, f.links, f.clov, p);
  return launched("k_dirac");
}

// Launch variants (threads per CTA, CTAs per SM the register budget must
// allow): (128, 5) ~100 registers, (128, 6) ~80, (256, 2) ~128 and (256, 3)
// ~85; for FP64 (128, 4) ~128, (128, 3) ~168, (256, 2) ~128, (256, 1) 255;
// variants 4-7 are 0-3 with the clover tiles read past L1.
// A 256-thread CTA covers one whole 4^4 block, so interior neighbours are
// read by the same SM.
constexpr int DIRAC_VARIANTS = 8;

template <typename S, typename SO = S>
int dirac_t(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st) {
  auto shape = [&](int v, auto nl1) {
    constexpr bool N = decltype(nl1)::value;
    if constexpr (Store<S>::prec == DD_F64 || Store<S>::prec == DD_PREC_DF) {
      // FP64 and double-float values take two registers each: looser caps
      switch (v) {
        case 1: return dirac_v<S, 128, 3, N, SO>(g, f, p, st);
        case 2: return dirac_v<S, 256, 2, N, SO>(g, f, p, st);
        case 3: return dirac_v<S, 256, 1, N, SO>(g, f, p, st);
        default: return dirac_v<S, 128, 4, N, SO>(g, f, p, st);
      }
    } else {
      switch (v) {
        case 1: return dirac_v<S, 128, 6, N>(g, f, p, st);
        case 2: return dirac_v<S, 256, 2, N>(g, f, p, st);
        case 3: return dirac_v<S, 256, 3, N>(g, f, p, st);
        default: return dirac_v<S, 128, 5, N>(g, f, p, st);
      }
    }
  };
  auto run = [&](int v) {
    return v >= 4 ? shape(v - 4, std::true_type{}) : shape(v, std::false_type{});
  };
  int v = 0;
  int rc = tuned_variant(tune_key("dirac", g, f.prec, p.n), DIRAC_VARIANTS, run, st, &v);
  if (rc) return rc;
  return run(v);
}

}  // namespace

RhsPtrs contiguous(const void *in, void *out, int nrhs, size_t field_bytes) {
  RhsPtrs p;
  p.n = nrhs;
  for (int r = 0; r < nrhs && r < MAX_RHS; r++) {
    p.in[r] = (const char *)in + r * field_bytes;
    p.out[r] = (char *)out + r * field_bytes;
  }
  return p;
}

int launch_dirac(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st) {
  NvtxRange range("dd:dirac");
  if (p.n < 1 || p.n > MAX_RHS) {
    set_error("apply_D: 1..%d right-hand sides per launch", MAX_RHS);
    return DD_EINVAL;
  }
  switch (f.prec) {
    case DD_F64: return dirac_t<double>(g, f, p, st);
    case DD_F32: return dirac_t<float>(g, f, p, st);
    case DD_F16: return dirac_t<__half>(g, f, p, st);
    case DD_BF16: return dirac_t<__nv_bfloat16>(g, f, p, st);
    case DD_F16N: return dirac_t<hn16>(g, f, p, st);
  }
  set_error("apply_D: precision %d not available", f.prec);
  return DD_EINVAL;
}

int launch_dirac_df(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st) {
  if (p.n < 1 || p.n > MAX_RHS || f.prec != DD_PREC_DF || !f.links) {
    set_error("apply_D (double-float): double-float fields and 1..%d right-hand sides", MAX_RHS);
    return DD_EINVAL;
  }
  return dirac_t<dfs, double>(g, f, p, st);
}

int launch_dirac(const Geom &g, const OpFields &f, const void *in, void *out, int nrhs, cudaStream_t st) {
  const size_t fb = (size_t)g.V * spinor_site_bytes(f.prec);
  for (int r0 = 0; r0 < nrhs; r0 += MAX_RHS) {
    int n = nrhs - r0 < MAX_RHS ? nrhs - r0 : MAX_RHS;
    int rc = launch_dirac(g, f, contiguous((const char *)in + r0 * fb, (char *)out + r0 * fb, n, fb), st);
    if (rc) return rc;
  }
  return DD_OK;
}

}  // namespace dd
