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
template <typename S, int TPB, int MINB, int SHAPE, typename SO = S>
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
  clover_apply<S, C>(clov, g.Vb, b, s, x, acc);
  dirac_dir<0, S, C>(g, st, links, inr, acc);
  dirac_dir<1, S, C>(g, st, links, inr, acc);
  dirac_dir<2, S, C>(g, st, links, inr, acc);
  dirac_dir<3, S, C>(g, st, links, inr, acc);
  store_spinor<SO, C>(p.out[r], g, b, s, acc);
}

template <typename S, int TPB, int MINB, typename SO = S>
int dirac_v(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st) {
  long long n = g.V * p.n;
  const unsigned grid = (unsigned)((n + TPB - 1) / TPB);
  if (shape_of(g) == 1) k_dirac<S, TPB, MINB, 1, SO><<<grid, TPB, 0, st>>>(g, f.links, f.clov, p);
  else k_dirac<S, TPB, MINB, 0, SO><<<grid, TPB, 0, st>>>(g, f.links, f.clov, p);
  return launched("k_dirac");
}

// Launch variants (threads per CTA, CTAs per SM the register budget must
// allow): (128, 5) ~100 registers, (128, 6) ~80, (256, 2) ~128 and (256, 3)
// ~85; for FP64 (128, 4) ~128, (128, 3) ~168, (256, 2) ~128, (256, 1) 255.
// A 256-thread CTA covers one whole 4^4 block, so interior neighbours are
// read by the same SM.
constexpr int DIRAC_VARIANTS = 4;

template <typename S, typename SO = S>
int dirac_t(const Geom &g, const OpFields &f, const RhsPtrs &p, cudaStream_t st) {
  auto run = [&](int v) {
    if constexpr (Store<S>::prec == DD_F64 || Store<S>::prec == DD_PREC_DF) {
      // FP64 and double-float values take two registers each: looser caps
      switch (v) {
        case 1: return dirac_v<S, 128, 3, SO>(g, f, p, st);
        case 2: return dirac_v<S, 256, 2, SO>(g, f, p, st);
        case 3: return dirac_v<S, 256, 1, SO>(g, f, p, st);
        default: return dirac_v<S, 128, 4, SO>(g, f, p, st);
      }
    } else {
      switch (v) {
        case 1: return dirac_v<S, 128, 6>(g, f, p, st);
        case 2: return dirac_v<S, 256, 2>(g, f, p, st);
        case 3: return dirac_v<S, 256, 3>(g, f, p, st);
        default: return dirac_v<S, 128, 5>(g, f, p, st);
      }
    }
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
