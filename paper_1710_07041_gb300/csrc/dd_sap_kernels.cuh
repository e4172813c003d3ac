// Schwarz-kernel templates shared by the per-precision translation units
// (dd_sap_f64.cu, dd_sap_f32.cu, dd_sap_f16.cu, dd_sap_bf16.cu) and
// dd_sap.cu. See dd_sap.cu for the method.
#pragma once
#include <algorithm>
#include <functional>
#include <mutex>
#include <string>

#include "dd_tune.cuh"

namespace dd {

// device counter of expired bounded waits (resolved before any capture)
unsigned *sap_timeout_counter();
// run `enqueue` (the launches of one smoother application) as a cached CUDA graph
int sap_launch_as_graph(const std::string &key, int variant, int nkernels, const RhsPtrs &rp, const AuxPtrs *ax,
                        const std::function<int()> &enqueue, cudaStream_t st);

// Residual modes of one colour phase (bit set `mode` of k_sap_phase).
// Without SAP_INCR the phase forms r = b - D x on its blocks from x (b and x
// in HBM). With it, r = (b if SAP_FROM_B, else the block's stored residual
// after its own previous solve) minus, with SAP_HALO_E, the hops from the
// neighbouring blocks' latest corrections e: x changed only there since.
// SAP_WRITE_E / SAP_WRITE_R store this phase's corrections (as face flux
// where flux_layout holds, else e itself) and residuals for the next phases.
enum { SAP_INCR = 1, SAP_FROM_B = 2, SAP_HALO_E = 4, SAP_WRITE_E = 8, SAP_WRITE_R = 16 };

namespace {


// bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2
__device__ __forceinline__ void prefetch_l2(const void *gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

// ---- bulk (TMA) staging into shared memory, completion on an mbarrier
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
}
// the issuing thread's arrival, announcing `bytes` of bulk copies
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// one bulk copy global -> shared (addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// generic-proxy accesses of shared memory before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Bounded wait for phase `parity` of the staging barrier (shared address
// mbar): about one second of SM clock at most, then false.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;
__device__ __noinline__ bool mbar_wait_slow(unsigned mbar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_test(mbar, parity))
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
  return true;
}
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
  return mbar_test(mbar, parity) || mbar_wait_slow(mbar, parity);
}
// the CTA's wait expired: count it, let thread 0's copies land (bounded)
__device__ __noinline__ void wait_expired(unsigned *timeouts, unsigned mbar, unsigned parity) {
  if (threadIdx.x == 0) {
    atomicAdd(timeouts, 1u);
    mbar_wait_slow(mbar, parity);
  }
}

// ---- tensor memory (TMEM) as a per-thread store of the block's clover
// blocks (STAGE 3). TMEM has 128 lanes x 512 columns of 32 bits per SM; a
// warp reaches only the 32 lanes of its sub-partition (warp % 4), so thread
// t of the CTA owns lane t % 128 and a column range chosen by t / 128. Each
// clover block a thread multiplies with is read by that thread alone, which
// is the access TMEM allows. Allocation is per CTA (a power of two of at
// least 32 columns); the launch keeps at most 512 / NCOLS CTAs of TMEM
// kernels on an SM through their shared-memory size, so an allocation never
// waits for columns.
template <int NCOLS> __device__ __forceinline__ void tmem_alloc(unsigned dst_smem) {
  static_assert(NCOLS >= 32 && NCOLS <= 512 && (NCOLS & (NCOLS - 1)) == 0, "TMEM columns");
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "n"(NCOLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
template <int NCOLS> __device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "n"(NCOLS) : "memory");
}
// a CTA barrier that orders the threads' tensor-memory operations around it
__device__ __forceinline__ void tmem_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// the 36 reals of a clover block (m[0..17], real and imaginary parts in
// turn) to columns taddr ... taddr + 35 of the thread's lane (warp-collective)
__device__ __forceinline__ void tmem_st36(uint32_t taddr, const cpx<float> *m) {
  const float *f = (const float *)m;
  unsigned u[36];
#pragma unroll
  for (int i = 0; i < 36; i++) u[i] = __float_as_uint(f[i]);
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
      "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7]), "r"(u[8]), "r"(u[9]),
      "r"(u[10]), "r"(u[11]), "r"(u[12]), "r"(u[13]), "r"(u[14]), "r"(u[15]), "r"(u[16]), "r"(u[17]), "r"(u[18]),
      "r"(u[19]), "r"(u[20]), "r"(u[21]), "r"(u[22]), "r"(u[23]), "r"(u[24]), "r"(u[25]), "r"(u[26]), "r"(u[27]),
      "r"(u[28]), "r"(u[29]), "r"(u[30]), "r"(u[31])
      : "memory");
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(taddr + 32), "r"(u[32]),
               "r"(u[33]), "r"(u[34]), "r"(u[35])
               : "memory");
}
// the stores of this thread have landed (before the columns are read)
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// the inverse of tmem_st36 (warp-collective). Both loads and their wait are
// one asm statement: the destination registers are defined only after it.
__device__ __forceinline__ void tmem_ld36(uint32_t taddr, cpx<float> *m) {
  unsigned u[36];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%36];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%32, %33, %34, %35}, [%37];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
        "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
        "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31]), "=r"(u[32]),
        "=r"(u[33]), "=r"(u[34]), "=r"(u[35])
      : "r"(taddr), "r"(taddr + 32)
      : "memory");
  float *f = (float *)m;
#pragma unroll
  for (int i = 0; i < 36; i++) f[i] = __uint_as_float(u[i]);
}

// Strided view of one block's pair tile: pair-major (the links: element
// (i, site) at p[i * stride + site]) or chunked (the clover: see
// clover_block_chunked, stride = sites per chunk row).
template <typename P> struct Tile {
  const P *p;
  int stride;
};

// link mu of tile site s (all nine entries: the kernel reads the full-link
// field, OpFields::links_full)
template <typename C, typename P>
__device__ __forceinline__ void tile_link(const Tile<P> &t, int s, int mu, Link<C> &u) {
  DD_CHECK_INDEX(s, t.stride);
#pragma unroll
  for (int i = 0; i < 9; i++) u.m[i] = from_pair<C, P>(t.p[(9 * mu + i) * t.stride + s]);
}
// chirality block h of site s of a chunked clover tile (shared or global memory)
template <typename C, typename P>
__device__ __forceinline__ void tile_block(const Tile<P> &t, int s, int h, cpx<C> *m) {
  clover_block_chunked<false, C, P>(t.p, (size_t)t.stride, s, h, m);
}

// chirality block h of tile site s: from the thread's TMEM columns at taddr
// (STAGE 3, which stored exactly this block there) or from the tile
template <int STAGE, typename C, typename P>
__device__ __forceinline__ void clover_of(const Tile<P> &t, uint32_t taddr, int s, int h, cpx<C> *m) {
  if constexpr (STAGE == 3) tmem_ld36(taddr, m);
  else tile_block(t, s, h, m);
}

// shared-memory vector: [12][Vh] complex, one parity of the block
template <typename C>
__device__ __forceinline__ void vec_load(const cpx<C> *v, int Vh, int q, Spinor<C> &o) {
  DD_CHECK_INDEX(q, Vh);
#pragma unroll
  for (int i = 0; i < 12; i++) o.c[i] = v[i * Vh + q];
}

// In-block neighbours of one site for the two directions of its thread half:
// four 16-bit fields (dir 2h fwd, dir 2h bwd, dir 2h+1 fwd, dir 2h+1 bwd),
// each the neighbour's index within the other parity's half-vector, NONE if
// the hop leaves the block.
constexpr unsigned NONE = 0xFFFFu;
template <int MU, int DIR>
__device__ __forceinline__ unsigned inner_index(const Geom &g, const Site &t) {
  int nb, ns;
  float sg;
  bool inside;
  neighbour(g, t, MU, DIR, &nb, &ns, &sg, &inside);
  return inside ? (unsigned)(ns - (t.p ? 0 : g.Vh)) : NONE;
}
// (the directions are compile-time constants in each branch, so no Geom or
// Site array is indexed at run time)
__device__ __forceinline__ uint2 inner_neighbours(const Geom &g, const Site &t, int h) {
  if (h == 0)
    return make_uint2(inner_index<0, +1>(g, t) | (inner_index<0, -1>(g, t) << 16),
                      inner_index<1, +1>(g, t) | (inner_index<1, -1>(g, t) << 16));
  return make_uint2(inner_index<2, +1>(g, t) | (inner_index<2, -1>(g, t) << 16),
                    inner_index<3, +1>(g, t) | (inner_index<3, -1>(g, t) << 16));
}

// acc += hop pair in direction MU into the site at tile position s from the
// shared half-vector v (the other parity), links from tile L. nf/nbk: neighbour
// indices (NONE: outside the block); off: tile offset of the other parity.
// SW: acc holds its spin halves swapped.
template <int MU, bool SW, typename C, typename P>
__device__ __forceinline__ void hop_inner_dir(int Vh, int s, unsigned nf, unsigned nbk, int off, const cpx<C> *v,
                                              const Tile<P> &L, Spinor<C> &acc) {
  Link<C> u;
  Spinor<C> psi;
  if (nf != NONE) {
    vec_load(v, Vh, (int)nf, psi);
    tile_link(L, s, MU, u);
    hop<MU, true, C, SW>(acc, u, psi, (C)-0.5);
  }
  if (nbk != NONE) {
    vec_load(v, Vh, (int)nbk, psi);
    tile_link(L, (int)nbk + off, MU, u);
    hop<MU, false, C, SW>(acc, u, psi, (C)-0.5);
  }
}

// The thread's partial sum over its two directions, its own spin half h in
// acc.c[0..5] and the partner's half in acc.c[6..11] (exchange's layout).
template <typename C, typename P>
__device__ __forceinline__ void hops_inner(int Vh, int s, int h, uint2 nbr, int off, const cpx<C> *v,
                                           const Tile<P> &L, Spinor<C> &acc) {
#pragma unroll
  for (int i = 0; i < 12; i++) acc.c[i] = {0, 0};
  if (h == 0) {
    hop_inner_dir<0, false>(Vh, s, nbr.x & NONE, nbr.x >> 16, off, v, L, acc);
    hop_inner_dir<1, false>(Vh, s, nbr.y & NONE, nbr.y >> 16, off, v, L, acc);
  } else {
    hop_inner_dir<2, true>(Vh, s, nbr.x & NONE, nbr.x >> 16, off, v, L, acc);
    hop_inner_dir<3, true>(Vh, s, nbr.y & NONE, nbr.y >> 16, off, v, L, acc);
  }
}

// acc += hops into site t from the global field x, directions {2h, 2h+1};
// neighbours inside the block are skipped when self_zero (x known to be 0
// there), neighbours outside when halo_zero. SW: acc's spin halves swapped.
template <int MU, bool SW, typename S, typename C>
__device__ __forceinline__ void hop_global_dir(const Geom &g, const Site &t, const void *links, const void *x,
                                               bool self_zero, bool halo_zero, Spinor<C> &acc) {
  int nb, ns;
  float sg;
  bool inside;
  Link<C> u;
  Spinor<C> psi;
  neighbour(g, t, MU, +1, &nb, &ns, &sg, &inside);
  if (inside ? !self_zero : !halo_zero) {
    load_spinor<S, C>(x, g, nb, ns, psi);
    load_link<S, C, 9, false>(links, g, t.b, t.s, MU, u);
    hop<MU, true, C, SW>(acc, u, psi, (C)(-0.5f * sg));
  }
  neighbour(g, t, MU, -1, &nb, &ns, &sg, &inside);
  if (inside ? !self_zero : !halo_zero) {
    load_spinor<S, C>(x, g, nb, ns, psi);
    load_link<S, C, 9, false>(links, g, nb, ns, MU, u);
    hop<MU, false, C, SW>(acc, u, psi, (C)(-0.5f * sg));
  }
}

// (own spin half in acc.c[0..5], the partner's in acc.c[6..11], as hops_inner)
template <typename S, typename C>
__device__ __forceinline__ void hops_global(const Geom &g, const Site &t, int h, const void *links, const void *x,
                                            bool self_zero, bool halo_zero, Spinor<C> &acc) {
#pragma unroll
  for (int i = 0; i < 12; i++) acc.c[i] = {0, 0};
  if (h == 0) {
    hop_global_dir<0, false, S, C>(g, t, links, x, self_zero, halo_zero, acc);
    hop_global_dir<1, false, S, C>(g, t, links, x, self_zero, halo_zero, acc);
  } else {
    hop_global_dir<2, true, S, C>(g, t, links, x, self_zero, halo_zero, acc);
    hop_global_dir<3, true, S, C>(g, t, links, x, self_zero, halo_zero, acc);
  }
}

// ---- the face flux of a block's correction (SAP_HALO_E, flux layout).
// Halo entry q of a block: face f = 2 mu + (0: the block's upper face in mu,
// 1: its lower face), faces in order, and position k on the face (the three
// other directions in increasing order, the lowest fastest). When a block
// has solved for its correction e, it computes for each of its face sites x
// the hop of e(x) into the neighbouring block's site y = x +- mu and stores
// it at the entry of y (the opposite face, same position) in that block's
// part of the flux buffer: across its upper face W P e(x) with W =
// U_mu(x)^dagger, its own link; across its lower face only P e(x), whose
// link U_mu(y) belongs to the receiving block, which multiplies by it from
// its own tile. Both carry the antiperiodic sign. The receiving block reads
// its entries contiguously, instead of gathering e and the links of the
// neighbours at scattered sites; an entry is 6 complex (rows of two pairs).
__device__ __forceinline__ int face_area(const Geom &g, int mu) { return g.Vb >> g.lbd[mu]; }
__device__ __forceinline__ int halo_entries(const Geom &g) {
  return 2 * (face_area(g, 0) + face_area(g, 1) + face_area(g, 2) + face_area(g, 3));
}
__device__ __forceinline__ int face_offset(const Geom &g, int f) {
  int o = 0;
#pragma unroll
  for (int mu = 0; mu < 4; mu++) o += (2 * mu < f ? face_area(g, mu) : 0) + (2 * mu + 1 < f ? face_area(g, mu) : 0);
  return o;
}
// the flux layout: 32-bit arithmetic, and the buffer (6 complex per entry)
// fits in a spinor field of the lattice (true for blocks of extent >= 4)
template <typename C> __device__ __forceinline__ bool flux_layout(const Geom &g) {
  return sizeof(C) == 4 && halo_entries(g) <= 2 * g.Vb;
}
// entry q -> face f and position k on it
__device__ __forceinline__ void face_of(const Geom &g, int q, int &f, int &k) {
  f = 0;
  k = q;
#pragma unroll
  for (int ff = 0; ff < 7; ff++) {   // compile-time face directions
    const int a = face_area(g, ff >> 1);
    if (f == ff && k >= a) {
      k -= a;
      f++;
    }
  }
}
// the site at position k of face 2 MU + !UP of the block with coordinates
// bc (compile-time directions: no register array is indexed at run time)
template <int MU, bool UP> __device__ __forceinline__ Site face_site(const Geom &g, int b, const int *bc, int k) {
  constexpr int D0 = MU == 0 ? 1 : 0, D1 = MU <= 1 ? 2 : 1, D2 = MU <= 2 ? 3 : 2;
  Site t;
  t.b = b;
  t.lc[MU] = UP ? g.bd[MU] - 1 : 0;
  t.lc[D0] = k & (g.bd[D0] - 1);
  k >>= g.lbd[D0];
  t.lc[D1] = k & (g.bd[D1] - 1);
  t.lc[D2] = k >> g.lbd[D1];
  t.p = parity_of(t.lc);
  t.s = pos_of(g, t.lc);
#pragma unroll
  for (int d = 0; d < 4; d++) t.bc[d] = bc[d];
  return t;
}
// position on the face normal to MU of the site with local coordinates lc
template <int MU> __device__ __forceinline__ int face_pos(const Geom &g, const int *lc) {
  constexpr int D0 = MU == 0 ? 1 : 0, D1 = MU <= 1 ? 2 : 1, D2 = MU <= 2 ? 3 : 2;
  return lc[D0] + (lc[D1] << g.lbd[D0]) + (lc[D2] << (g.lbd[D0] + g.lbd[D1]));
}

template <typename P> struct alignas(2 * sizeof(P)) PairPair {
  P a, b;
};
// entry q of block bb: rows c = 0..2 of two pairs at ((bb * 3 + c) * E + q)
template <typename P, typename C>
__device__ __forceinline__ void flux_store(void *H, int E, int bb, int q, const cpx<C> *v) {
  PairPair<P> *p = (PairPair<P> *)H + (size_t)bb * 3 * E + q;
#pragma unroll
  for (int c = 0; c < 3; c++)
    p[(size_t)c * E] = {to_pair<P, C>(v[2 * c].re, v[2 * c].im), to_pair<P, C>(v[2 * c + 1].re, v[2 * c + 1].im)};
}
template <typename P, typename C>
__device__ __forceinline__ void flux_load(const void *H, int E, int bb, int q, cpx<C> *v) {
  const PairPair<P> *p = (const PairPair<P> *)H + (size_t)bb * 3 * E + q;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const PairPair<P> w = p[(size_t)c * E];
    v[2 * c] = from_pair<C, P>(w.a);
    v[2 * c + 1] = from_pair<C, P>(w.b);
  }
}

// Entry k of face 2 MU + !UP of block b (coordinates bc) as producer: the
// flux of e(x) into the neighbouring block's entry (see above)
template <int MU, bool UP, typename S, typename C, typename P>
__device__ __forceinline__ void flux_produce_entry(const Geom &g, int b, const int *bc, int k, const Tile<P> &Lt,
                                                   const cpx<C> *ve, const cpx<C> *vo, int E, void *H) {
  const Site t = face_site<MU, UP>(g, b, bc, k);
  int nb, ns;
  float sg;
  bool inside;
  neighbour(g, t, MU, UP ? +1 : -1, &nb, &ns, &sg, &inside);
  Spinor<C> ev;
  vec_load(t.p ? vo : ve, g.Vh, t.s - t.p * g.Vh, ev);
  cpx<C> chi[6], out[6];
  project<MU, !UP>(ev, chi);
  if constexpr (UP) {
    Link<C> u;
    cpx<C> hv[6];
    tile_link(Lt, t.s, MU, u);
    su3_dmul(u, chi, hv);
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = {(C)sg * hv[i].re, (C)sg * hv[i].im};
  } else {
#pragma unroll
    for (int i = 0; i < 6; i++) out[i] = {(C)sg * chi[i].re, (C)sg * chi[i].im};
  }
  // the receiving entry: the opposite face, same position
  flux_store<P>(H, E, nb, face_offset(g, 2 * MU + (UP ? 1 : 0)) + k, out);
}
// A block's correction (even sites in ve, odd sites in vo: [12][Vh] shared
// vectors) into the flux buffer H of its neighbours, one entry per thread
// at a time.
template <typename S, typename C, typename P>
__device__ __forceinline__ void flux_produce(const Geom &g, int b, const int *bc, const Tile<P> &Lt, const cpx<C> *ve,
                                             const cpx<C> *vo, void *H) {
  const int E = halo_entries(g);
#pragma unroll 1
  for (int q = threadIdx.x; q < E; q += blockDim.x) {
    int f, k;
    face_of(g, q, f, k);
    switch (f) {   // uniform across a warp where faces hold whole warps of entries
      case 0: flux_produce_entry<0, true, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      case 1: flux_produce_entry<0, false, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      case 2: flux_produce_entry<1, true, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      case 3: flux_produce_entry<1, false, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      case 4: flux_produce_entry<2, true, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      case 5: flux_produce_entry<2, false, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      case 6: flux_produce_entry<3, true, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
      default: flux_produce_entry<3, false, S>(g, b, bc, k, Lt, ve, vo, E, H); break;
    }
  }
}
// entry q (face 2 MU + !UP, position k) as receiver: the upper faces'
// projections multiplied by this block's link U_mu(y)
template <int MU, bool UP, typename C, typename P>
__device__ __forceinline__ void flux_receive_entry(const Geom &g, int k, int q, int E, const Tile<P> &Lt,
                                                   const void *H, int b, cpx<C> *hs) {
  cpx<C> v[6];
  flux_load<P>(H, E, b, q, v);
  if constexpr (UP) {
    constexpr int D0 = MU == 0 ? 1 : 0, D1 = MU <= 1 ? 2 : 1, D2 = MU <= 2 ? 3 : 2;
    int lc[4];
    lc[MU] = g.bd[MU] - 1;
    lc[D0] = k & (g.bd[D0] - 1);
    k >>= g.lbd[D0];
    lc[D1] = k & (g.bd[D1] - 1);
    lc[D2] = k >> g.lbd[D1];
    Link<C> u;
    cpx<C> hv[6];
    tile_link(Lt, pos_of(g, lc), MU, u);
    su3_mul(u, v, hv);
#pragma unroll
    for (int i = 0; i < 6; i++) v[i] = hv[i];
  }
#pragma unroll
  for (int i = 0; i < 6; i++) hs[i * E + q] = v[i];
}
// The block's incoming flux into hs (shared, [6][E] complex); ends with a
// barrier.
template <typename S, typename C, typename P>
__device__ __forceinline__ void flux_receive(const Geom &g, int b, const Tile<P> &Lt, const void *H, cpx<C> *hs) {
  const int E = halo_entries(g);
#pragma unroll 1
  for (int q = threadIdx.x; q < E; q += blockDim.x) {
    int f, k;
    face_of(g, q, f, k);
    switch (f) {
      case 0: flux_receive_entry<0, true>(g, k, q, E, Lt, H, b, hs); break;
      case 1: flux_receive_entry<0, false>(g, k, q, E, Lt, H, b, hs); break;
      case 2: flux_receive_entry<1, true>(g, k, q, E, Lt, H, b, hs); break;
      case 3: flux_receive_entry<1, false>(g, k, q, E, Lt, H, b, hs); break;
      case 4: flux_receive_entry<2, true>(g, k, q, E, Lt, H, b, hs); break;
      case 5: flux_receive_entry<2, false>(g, k, q, E, Lt, H, b, hs); break;
      case 6: flux_receive_entry<3, true>(g, k, q, E, Lt, H, b, hs); break;
      default: flux_receive_entry<3, false>(g, k, q, E, Lt, H, b, hs); break;
    }
  }
  __syncthreads();
}

// acc (spin half h of a site) += sgn * that half of reconstruct(hv)
template <int MU, bool FWD, typename C>
__device__ __forceinline__ void recon_half(cpx<C> *acc, const cpx<C> *hv, int h, C sgn) {
  if (h == 0) {
#pragma unroll
    for (int i = 0; i < 6; i++) {
      acc[i].re = mad(sgn, hv[i].re, acc[i].re);
      acc[i].im = mad(sgn, hv[i].im, acc[i].im);
    }
    return;
  }
  const C s = FWD ? -sgn : sgn;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<C> h0 = hv[c], h1 = hv[3 + c];
    cpx<C> &l0 = acc[c], &l1 = acc[3 + c];
    if constexpr (MU == 0) {
      l0.re = mad(-s, h1.im, l0.re); l0.im = mad(s, h1.re, l0.im);
      l1.re = mad(-s, h0.im, l1.re); l1.im = mad(s, h0.re, l1.im);
    } else if constexpr (MU == 1) {
      l0.re = mad(s, h1.re, l0.re); l0.im = mad(s, h1.im, l0.im);
      l1.re = mad(-s, h0.re, l1.re); l1.im = mad(-s, h0.im, l1.im);
    } else if constexpr (MU == 2) {
      l0.re = mad(-s, h0.im, l0.re); l0.im = mad(s, h0.re, l0.im);
      l1.re = mad(s, h1.im, l1.re); l1.im = mad(-s, h1.re, l1.im);
    } else {
      l0.re = mad(s, h0.re, l0.re); l0.im = mad(s, h0.im, l0.im);
      l1.re = mad(s, h1.re, l1.re); l1.im = mad(s, h1.im, l1.im);
    }
  }
}
// the entry of site t's face in direction MU, if t lies on one
template <int MU, typename C>
__device__ __forceinline__ void flux_gather_dir(const Geom &g, const Site &t, int h, int E, const cpx<C> *hs,
                                                cpx<C> *acc) {
  const bool up = t.lc[MU] == g.bd[MU] - 1, lo = t.lc[MU] == 0;
  if (!up && !lo) return;
  const int q = face_offset(g, 2 * MU + (up ? 0 : 1)) + face_pos<MU>(g, t.lc);
  cpx<C> hv[6];
#pragma unroll
  for (int i = 0; i < 6; i++) hv[i] = hs[i * E + q];
  if (up) recon_half<MU, true>(acc, hv, h, (C)-0.5);
  else recon_half<MU, false>(acc, hv, h, (C)-0.5);
}
// r (spin half h of the thread's even and odd site) -= the incoming hops
template <typename C>
__device__ __forceinline__ void flux_gather(const Geom &g, const Site &se, const Site &so, int h, const cpx<C> *hs,
                                            cpx<C> *r_e, cpx<C> *r_o) {
  const int E = halo_entries(g);
  cpx<C> acc[6];
#pragma unroll
  for (int i = 0; i < 6; i++) acc[i] = {0, 0};
  flux_gather_dir<0>(g, se, h, E, hs, acc);
  flux_gather_dir<1>(g, se, h, E, hs, acc);
  flux_gather_dir<2>(g, se, h, E, hs, acc);
  flux_gather_dir<3>(g, se, h, E, hs, acc);
#pragma unroll
  for (int i = 0; i < 6; i++) {
    r_e[i].re -= acc[i].re;
    r_e[i].im -= acc[i].im;
    acc[i] = {0, 0};
  }
  flux_gather_dir<0>(g, so, h, E, hs, acc);
  flux_gather_dir<1>(g, so, h, E, hs, acc);
  flux_gather_dir<2>(g, so, h, E, hs, acc);
  flux_gather_dir<3>(g, so, h, E, hs, acc);
#pragma unroll
  for (int i = 0; i < 6; i++) {
    r_o[i].re -= acc[i].re;
    r_o[i].im -= acc[i].im;
  }
}

// the six components of spin half h (selects, so the register arrays are
// never indexed at run time)
template <typename C>
__device__ __forceinline__ void half_of(const Spinor<C> &s, int h, cpx<C> *out) {
#pragma unroll
  for (int i = 0; i < 6; i++) out[i] = h ? s.c[6 + i] : s.c[i];
}

// Exchange partial hop sums between the two halves of a site pair (part:
// own spin half h in c[0..5], the partner's in c[6..11]): on return
// own[0..5] = full sum of the components of half h. xch: [12][Vh] smem. A
// thread reads only the entries its partner wrote for it, so the next write
// to xch needs one barrier after this call (every caller has one).
template <typename C>
__device__ __forceinline__ void exchange(cpx<C> *xch, int Vh, int j, int h, const Spinor<C> &part, cpx<C> *own) {
  const int other = 6 * (1 - h), mine = 6 * h;
#pragma unroll
  for (int i = 0; i < 6; i++) xch[(other + i) * Vh + j] = part.c[6 + i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 6; i++) {
    cpx<C> a = part.c[i], b = xch[(mine + i) * Vh + j];
    own[i] = {a.re + b.re, a.im + b.im};
  }
}

// deterministic block sum of three values; red: smem [3][32]. NW: warps per
// CTA when the block shape fixes it at compile time (whole warps), else 0
// (any blockDim.x up to 1024). The reads of red are not followed by a barrier
// here: the caller reaches one (the end of its half-step) before any thread
// can write red again.
template <int NW, typename C>
__device__ __forceinline__ void block_sum3(C &a, C &b, C &c, C *red) {
  static_assert(NW >= 0 && NW <= 32, "warps per CTA");
  const int width = NW > 0 ? 32 : (blockDim.x < 32 ? blockDim.x : 32);
  const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (o < width) {
      a += __shfl_xor_sync(mask, a, o);
      b += __shfl_xor_sync(mask, b, o);
      c += __shfl_xor_sync(mask, c, o);
    }
  }
  const int w = threadIdx.x / 32, nw = NW > 0 ? NW : (blockDim.x + 31) / 32;
  if ((threadIdx.x & 31) == 0) {
    red[w] = a;
    red[32 + w] = b;
    red[64 + w] = c;
  }
  __syncthreads();
  a = b = c = 0;
#pragma unroll
  for (int i = 0; i < (NW > 0 ? NW : 32); i++) {
    if (NW == 0 && i >= nw) break;
    a += red[i];
    b += red[32 + i];
    c += red[64 + i];
  }
}

template <typename S> struct SapSmem {
  using C = typename Store<S>::comp_t;
  using P = typename Store<S>::pair_t;
  static constexpr int LT = 36;   // pairs per site of the links tile (full links)
  static size_t vec_bytes(const Geom &g) { return (size_t)12 * g.Vh * sizeof(cpx<C>); }
  // TMEM columns of a STAGE-3 CTA: 128 per group of 128 threads (its A_ee^-1
  // block at +0, its A_oo block at +64)
  static int tmem_cols(const Geom &g) { return g.Vb > 256 ? 512 : 256; }
  // stage: 0 nothing staged, 1 links + A_oo + A_ee^-1, 2 links only, 3 links
  // staged and the clover blocks in TMEM (at least 80 KB, or 150 KB with 512
  // columns: of an SM's 228 KB, two 256-column CTAs fit, three do not, nor
  // a 512-column CTA beside any other)
  static size_t bytes(const Geom &g, int stage) {
    size_t b = 3 * vec_bytes(g) + 96 * sizeof(C) + 16;   // + staging mbarrier, TMEM address
    if (stage == 1) b += ((size_t)LT * g.Vb + (size_t)36 * 2 * g.Vh) * sizeof(P);
    if (stage == 2 || stage == 3) b += (size_t)LT * g.Vb * sizeof(P);
    if (stage == 3) b = std::max(b, (size_t)(tmem_cols(g) > 256 ? 150 : 80) * 1024);
    return b;
  }
};

// The group of work item `item` (groups in item order).
__device__ __forceinline__ int sap_group_of(const SapGroups &G, int item) {
  int k = 0;
#pragma unroll 1
  while (k + 1 < G.n && item >= G.grp[k + 1].item0) k++;
  return k;
}
// the i-th block of colour `colour`: blocks 2i and 2i+1 differ in colour
__device__ __forceinline__ int sap_block_of(const Geom &g, int colour, int bi) {
  int bb = 2 * bi, bc[4];
  block_coords(g, bb, bc);
  return (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) ? bb + 1 : bb;
}

// STAGE: 0 operator tiles read through L1/L2; 1 links, A_oo and A_ee^-1 staged
// in shared memory; 2 links staged, the clover blocks (each read by one
// thread only) through L1/L2, which halves the footprint. UNROLL (specialised
// shapes only): the MR loop's even and odd half-steps as separate code.
// MULTI: the launch covers several lattice groups (without it, group 0 only,
// whose fields the compiler reads at constant offsets).
template <typename S, int STAGE, int MINB, int NT, int SHAPE, bool UNROLL = false, bool MULTI = false>
__global__ void __launch_bounds__(NT, MINB) k_sap_phase(const SapGroups G, const RhsPtrs rp, const AuxPtrs ax,
                                                   int colour, int self_zero, int halo_zero, int mode, int nmr,
                                                   int tile, unsigned *timeouts) {
  using C = typename Store<S>::comp_t;
  using P = typename Store<S>::pair_t;
  constexpr int LT = SapSmem<S>::LT;   // pairs per site of the links tile
  // a specialised shape is launched with one thread per site: blockDim.x == NT
  static_assert(SHAPE == 0 || (SHAPE == 1 && NT == 256) || (SHAPE == 2 && NT == 512), "shape / threads");
  // TMEM holds FP32 clover blocks, one thread per lane: specialised shapes only
  static_assert(STAGE != 3 || (SHAPE != 0 && sizeof(C) == 4), "TMEM clover: FP32 arithmetic, fixed shape");
  constexpr int TCOLS = NT > 256 ? 512 : 256;
  extern __shared__ __align__(16) unsigned char smem[];
  // every group of a launch has the same block shape (checked on the host)
  const int Vh = block_shape<SHAPE>(G.grp[0].g).Vh, Vb = block_shape<SHAPE>(G.grp[0].g).Vb;
  const int h = threadIdx.x / Vh, j = threadIdx.x - h * Vh;

  cpx<C> *rho = (cpx<C> *)smem;   // MR residual on odd sites (then e_o)
  cpx<C> *te = rho + 12 * Vh;     // even-site temporary
  cpx<C> *xch = te + 12 * Vh;     // partial-sum exchange between thread halves
  C *red = (C *)(xch + 12 * Vh);
  uint64_t *mbar = (uint64_t *)(red + 96);   // staging barrier (16 bytes reserved)
  uint32_t *tmem_at = (uint32_t *)(mbar + 1);  // TMEM base address (STAGE 3)
  unsigned char *tiles = (unsigned char *)(red + 96) + 16;
  unsigned phase = 0;                        // parity of the staging barrier's current phase
  if constexpr (STAGE != 0) {
    if (threadIdx.x == 0) mbar_init(mbar);
    if constexpr (STAGE == 3) {
      if (threadIdx.x < 32) tmem_alloc<TCOLS>(smem_u32(tmem_at));
      tmem_sync();
    } else {
      __syncthreads();
    }
  }
  const unsigned mbar_s = smem_u32(mbar);
  // this thread's TMEM columns: lane threadIdx.x % 128 (the warp's
  // sub-partition), 128 columns per group of 128 threads
  uint32_t tm = 0;
  if constexpr (STAGE == 3)
    tm = *tmem_at + ((uint32_t)(32 * ((threadIdx.x / 32) % 4)) << 16) + (uint32_t)(threadIdx.x / 128) * 128u;
  bool quit = false;   // a staging wait expired: leave through the common exit

  // Work items: (lattice group, block of this colour, right-hand-side tile),
  // block fastest within a group; group k holds items G.grp[k].item0 ... A
  // CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ...; while it works
  // on one, the next one's operator tiles and fields are prefetched into L2.
  // one lattice: its geometry and fields once, outside the item loop
  const Geom g0 = block_shape<SHAPE>(G.grp[0].g);
#pragma unroll 1
  for (int item = blockIdx.x; item < G.nitems; item += gridDim.x) {
  const int k = MULTI ? sap_group_of(G, item) : 0;
  const Geom g = MULTI ? block_shape<SHAPE>(G.grp[k].g) : g0;
  const void *__restrict__ links = G.grp[k].links;
  const void *__restrict__ clov = G.grp[k].clov;
  const void *__restrict__ cinv = G.grp[k].cinv;
  const int nbc = g.nblocks / 2, rhs0 = MULTI ? G.grp[k].rhs0 : 0, nrhs = MULTI ? G.grp[k].nrhs : rp.n;
  const int loc = MULTI ? item - G.grp[k].item0 : item;
  const int b = sap_block_of(g, colour, loc % nbc), rt = loc / nbc;
  if (threadIdx.x == 0) {
    // this item's own fields that are read later in its lifetime (x at the
    // end, the stored residual and the incoming flux after the operator's
    // staging), requested into L2 now; with one CTA per block nothing else
    // prefetches them
    constexpr unsigned SB = (unsigned)spinor_site_bytes(Store<S>::prec);
    constexpr int NC = spinor_chunks<S>();
    const size_t off = (size_t)b * Vb * SB;
    for (int q = 0; q < tile; q++) {
      const int r = rt * tile + q;
      if (r >= nrhs) break;
      if (!self_zero) prefetch_l2((const char *)rp.out[rhs0 + r] + off, Vb * SB);
      if ((mode & SAP_INCR) && !(mode & SAP_FROM_B))
        for (int c = 0; c < NC; c++) prefetch_l2((const char *)ax.r[rhs0 + r] + off + ((size_t)c * Vb + Vh) * 16, Vh * 16u);
      if (sizeof(C) == 4 && (mode & SAP_INCR) && (mode & SAP_HALO_E) && flux_layout<C>(g)) {
        const unsigned fb = 3u * halo_entries(g) * sizeof(PairPair<P>);
        prefetch_l2((const char *)ax.e[rhs0 + r] + (size_t)b * fb, fb);
      }
    }
  }
  if (threadIdx.x == 0 && item + (int)gridDim.x < G.nitems) {
    const int nitem = item + gridDim.x, nk = MULTI ? sap_group_of(G, nitem) : 0;
    const Geom ng = MULTI ? block_shape<SHAPE>(G.grp[nk].g) : g0;
    const int nnbc = ng.nblocks / 2, nloc = MULTI ? nitem - G.grp[nk].item0 : nitem;
    const int nb = sap_block_of(ng, colour, nloc % nnbc), nrt = nloc / nnbc;
    // exactly what the item reads: the incremental modes read the clover
    // only on odd sites (A_oo) and, after the first sweep, the stored
    // residual on odd sites instead of b (16-byte pieces of Vh sites per
    // chunk row)
    const bool incr = mode & SAP_INCR, from_b = !incr || (mode & SAP_FROM_B);
    constexpr int CP = chunk_pairs<P>(), NC = spinor_chunks<S>();
    prefetch_l2((const P *)G.grp[nk].links + (size_t)nb * LT * Vb, (unsigned)LT * Vb * sizeof(P));
    const P *nclov = (const P *)G.grp[nk].clov + (size_t)nb * 36 * Vb;
    if (incr) {
      for (int c = 0; c < 36 / CP; c++) prefetch_l2(nclov + ((size_t)c * Vb + Vh) * CP, Vh * 16u);
    } else {
      prefetch_l2(nclov, 36u * Vb * sizeof(P));
    }
    prefetch_l2((const P *)G.grp[nk].cinv + (size_t)nb * 36 * Vh, 36u * Vh * sizeof(P));
    const int nrhs0 = MULTI ? G.grp[nk].rhs0 : 0, nnrhs = MULTI ? G.grp[nk].nrhs : rp.n;
    for (int q = 0; q < tile; q++) {
      const int r = nrt * tile + q;
      if (r >= nnrhs) break;
      // a block of a spinor field: NC chunk rows of Vb x 16 bytes (then, for
      // DD_F16N, Vb FP32 scales), contiguous
      constexpr unsigned SB = (unsigned)spinor_site_bytes(Store<S>::prec);
      const size_t off = (size_t)nb * Vb * SB;
      if (from_b) prefetch_l2((const char *)rp.in[nrhs0 + r] + off, Vb * SB);
      else
        for (int c = 0; c < NC; c++) prefetch_l2((const char *)ax.r[nrhs0 + r] + off + ((size_t)c * Vb + Vh) * 16, Vh * 16u);
      if (!self_zero) prefetch_l2((const char *)rp.out[nrhs0 + r] + off, Vb * SB);
    }
  }

  // Staging by bulk copies (the TMA engine), issued by thread 0 and tracked
  // by the mbarrier: the links tile (LT x Vb pairs, contiguous per block),
  // and for STAGE 1 the odd half of every clover chunk row (36 / CP pieces of
  // Vh chunks) and the even-site inverse tile (contiguous). Every size is a
  // multiple of 16 bytes and every address 16-byte aligned.
  Tile<P> Lt, Ao, Ai;
  if constexpr (STAGE == 1) {
    P *sl = (P *)tiles;
    P *sa = sl + (size_t)LT * Vb;
    P *si = sa + (size_t)36 * Vh;
    if (threadIdx.x == 0) {
      constexpr int CP = chunk_pairs<P>();
      const P *gl = (const P *)links + (size_t)b * LT * Vb;
      const P *ga = (const P *)clov + (size_t)b * 36 * Vb;
      const unsigned lb = (unsigned)LT * Vb * sizeof(P), rb = (unsigned)(Vh * 16);
      fence_proxy_async();
      mbar_arrive_expect(mbar, lb + 2u * (36 / CP) * rb);
      bulk_g2s(sl, gl, lb, mbar);
      for (int c = 0; c < 36 / CP; c++)
        bulk_g2s(sa + (size_t)c * Vh * CP, ga + ((size_t)c * Vb + Vh) * CP, rb, mbar);
      bulk_g2s(si, (const P *)cinv + (size_t)b * 36 * Vh, (36u / CP) * rb, mbar);
    }
    Lt = {sl, Vb};
    Ao = {sa, Vh};
    Ai = {si, Vh};
  } else if constexpr (STAGE == 2 || STAGE == 3) {
    P *sl = (P *)tiles;
    if (threadIdx.x == 0) {
      const unsigned lb = (unsigned)LT * Vb * sizeof(P);
      fence_proxy_async();
      mbar_arrive_expect(mbar, lb);
      bulk_g2s(sl, (const P *)links + (size_t)b * LT * Vb, lb, mbar);
    }
    Lt = {sl, Vb};
    Ao = {(const P *)clov + (size_t)b * 36 * Vb + (size_t)Vh * chunk_pairs<P>(), Vb};
    Ai = {(const P *)cinv + (size_t)b * 36 * Vh, Vh};
  } else {
    Lt = {(const P *)links + (size_t)b * LT * Vb, Vb};
    Ao = {(const P *)clov + (size_t)b * 36 * Vb + (size_t)Vh * chunk_pairs<P>(), Vb};
    Ai = {(const P *)cinv + (size_t)b * 36 * Vh, Vh};
  }

  if constexpr (STAGE == 3) {
    // this thread's two clover blocks (A_ee^-1 of even site j, A_oo of odd
    // site j, chirality h) into its TMEM columns; the previous item's reads
    // of them completed (tmem_ld36 waits). Both blocks are loaded before the
    // first store (one round trip to L2 per item, not two).
    cpx<C> mi[18], mo[18];
    tile_block(Ai, j, h, mi);
    tile_block(Ao, j, h, mo);
    tmem_st36(tm, mi);
    tmem_st36(tm + 64, mo);
    tmem_wait_st();
  }
  const Site se = decode(g, b, j), so = decode(g, b, Vh + j);
  const uint2 nbr_e = inner_neighbours(g, se, h), nbr_o = inner_neighbours(g, so, h);
  // corrections travel between phases as face flux (32-bit arithmetic,
  // blocks whose flux fits a spinor field; the same for every phase of the
  // lattice), else as e itself
  const bool flux = flux_layout<C>(g);
  // the flux receiver multiplies by the staged links: wait for them first
  const bool early = flux && (mode & SAP_INCR) && (mode & SAP_HALO_E);
  // right-hand sides blockIdx.y * tile ... share the staged tiles
#pragma unroll 1
  for (int rr = 0; rr < tile; rr++) {
    if (rt * tile + rr >= nrhs) break;
    const int r = rhs0 + rt * tile + rr;
    const void *bf = rp.in[r];
    void *xf = rp.out[r];
    cpx<C> r_e[6], r_o[6];
    if constexpr (STAGE != 0) {
      // the staging of this item completes phase `phase` of the barrier;
      // a CTA whose wait expired leaves as a whole (the flag is raised)
      if (rr == 0 && early) {
        const bool ok = mbar_wait(mbar_s, phase);
        if (__syncthreads_or(!ok)) {
          wait_expired(timeouts, mbar_s, phase);
          quit = true;
          break;
        }
        phase ^= 1u;
      }
    }
    if constexpr (sizeof(C) == 4)
      if (early) flux_receive<S, C, P>(g, b, Lt, ax.e[r], rho);

    // ---- 2. block residual (halves h of the even and odd site): r = b - D x,
    // or incrementally (SAP_INCR) from the stored residual and the hops of
    // the neighbours' corrections across the block faces
    if ((mode & SAP_INCR) && !(mode & SAP_FROM_B)) {
      Spinor<C> rs;
      load_spinor<S, C>(ax.r[r], g, b, Vh + j, rs);
      half_of(rs, h, r_o);
  #pragma unroll
      for (int i = 0; i < 6; i++) r_e[i] = {0, 0};
    } else {
      Spinor<C> bb;
      load_spinor<S, C>(bf, g, b, j, bb);
      half_of(bb, h, r_e);
      load_spinor<S, C>(bf, g, b, Vh + j, bb);
      half_of(bb, h, r_o);
    }
    if (mode & SAP_INCR) {
      if (early) {
        flux_gather(g, se, so, h, rho, r_e, r_o);
        __syncthreads();
      } else if (mode & SAP_HALO_E) {
  #pragma unroll 1
        for (int par = 0; par < 2; par++) {
          Spinor<C> part;
          hops_global<S, C>(g, par ? so : se, h, links, ax.e[r], true, false, part);
          cpx<C> hx[6];
          exchange(xch, Vh, j, h, part, hx);
  #pragma unroll
          for (int i = 0; i < 6; i++) {
            if (par) { r_o[i].re -= hx[i].re; r_o[i].im -= hx[i].im; }
            else     { r_e[i].re -= hx[i].re; r_e[i].im -= hx[i].im; }
          }
          __syncthreads();
        }
      }
    } else if (!(self_zero && halo_zero)) {
  #pragma unroll 1
      for (int par = 0; par < 2; par++) {
        const Site &t = par ? so : se;
        Spinor<C> part;
        hops_global<S, C>(g, t, h, links, xf, self_zero, halo_zero, part);
        cpx<C> hx[6], ax[6] = {}, m[18], xh[6];
        exchange(xch, Vh, j, h, part, hx);
        if (!self_zero) {
          Spinor<C> xs;
          load_spinor<S, C>(xf, g, b, t.s, xs);
          half_of(xs, h, xh);
          load_clover_block<S, C>(clov, Vb, b, t.s, h, m);
          herm6_mv(m, xh, ax);
        }
  #pragma unroll
        for (int i = 0; i < 6; i++) {
          cpx<C> d = {ax[i].re + hx[i].re, ax[i].im + hx[i].im};
          if (par) { r_o[i].re -= d.re; r_o[i].im -= d.im; }
          else     { r_e[i].re -= d.re; r_e[i].im -= d.im; }
        }
        __syncthreads();
      }
    }
    if constexpr (STAGE != 0) {
      if (rr == 0 && !early) {
        const bool ok = mbar_wait(mbar_s, phase);
        if (__syncthreads_or(!ok)) {
          wait_expired(timeouts, mbar_s, phase);
          quit = true;
          break;
        }
        phase ^= 1u;
      }
    }

    // ---- 3.-5. Schur right-hand side, MR steps, reconstruction: half-steps,
    // odd steps on the odd site (input te), even steps on the even site
    // (input rho). Step 0: rho = r_o - D_oe A_ee^-1 r_e. Steps 1..2 n_MR:
    // te = A_ee^-1 D_eo rho, then p = A_oo rho - D_oe te and the MR update.
    // Last step: e_e = A_ee^-1 (r_e - D_eo e_o).
    cpx<C> m[18], tmp[6], rh[6], eo[6], ee[6];
    clover_of<STAGE>(Ai, tm, j, h, m);
    herm6_mv(m, r_e, tmp);
  #pragma unroll
    for (int i = 0; i < 6; i++) {
      te[(6 * h + i) * Vh + j] = tmp[i];
      eo[i] = {0, 0};
      rh[i] = {0, 0};
    }
    __syncthreads();
    // step 0: rho = r_o - D_oe te (no clover multiply: rho is still zero)
    {
      Spinor<C> part;
      hops_inner(Vh, Vh + j, h, nbr_o, 0, te, Lt, part);
      cpx<C> hv[6];
      exchange(xch, Vh, j, h, part, hv);
  #pragma unroll
      for (int i = 0; i < 6; i++) {
        rh[i] = {r_o[i].re - hv[i].re, r_o[i].im - hv[i].im};
        rho[(6 * h + i) * Vh + j] = nmr == 0 ? eo[i] : rh[i];
      }
      __syncthreads();
    }
    if constexpr (UNROLL && SHAPE != 0) {
    // steps 2k-1 (even) and 2k (odd) for k = 1..n_MR as separate code, then
    // the last even step: no run-time parity selects, twice the hop code
  #pragma unroll 1
    for (int k = 1; k <= nmr + 1; k++) {
      const bool last = k == nmr + 1;
      {   // even: te = A_ee^-1 D_eo rho, or on the last step e_e = A_ee^-1 (r_e - D_eo e_o)
        Spinor<C> part;
        hops_inner(Vh, j, h, nbr_e, Vh, rho, Lt, part);
        cpx<C> hv[6], u[6], mu[6];
        exchange(xch, Vh, j, h, part, hv);
  #pragma unroll
        for (int i = 0; i < 6; i++) u[i] = last ? cpx<C>{r_e[i].re - hv[i].re, r_e[i].im - hv[i].im} : hv[i];
        clover_of<STAGE>(Ai, tm, j, h, m);
        herm6_mv(m, u, mu);
        if (last) {
  #pragma unroll
          for (int i = 0; i < 6; i++) ee[i] = mu[i];
        } else {
  #pragma unroll
          for (int i = 0; i < 6; i++) te[(6 * h + i) * Vh + j] = mu[i];
        }
        __syncthreads();
      }
      if (last) break;
      {   // odd: p = A_oo rho - D_oe te and the MR update of e_o and rho
        Spinor<C> part;
        hops_inner(Vh, Vh + j, h, nbr_o, 0, te, Lt, part);
        cpx<C> hv[6], mu[6], p[6];
        exchange(xch, Vh, j, h, part, hv);
        clover_of<STAGE>(Ao, tm + 64, j, h, m);
        herm6_mv(m, rh, mu);
        C pr_re = 0, pr_im = 0, pp = 0;
  #pragma unroll
        for (int i = 0; i < 6; i++) {
          p[i] = {mu[i].re - hv[i].re, mu[i].im - hv[i].im};
          pr_re += p[i].re * rh[i].re + p[i].im * rh[i].im;
          pr_im += p[i].re * rh[i].im - p[i].im * rh[i].re;
          pp += p[i].re * p[i].re + p[i].im * p[i].im;
        }
        block_sum3<SHAPE != 0 ? NT / 32 : 0>(pr_re, pr_im, pp, red);
        C a_re = 0, a_im = 0;
        if (pp > (C)0) {
          a_re = pr_re / pp;
          a_im = pr_im / pp;
        }
  #pragma unroll
        for (int i = 0; i < 6; i++) {
          eo[i].re += a_re * rh[i].re - a_im * rh[i].im;
          eo[i].im += a_re * rh[i].im + a_im * rh[i].re;
          rh[i].re -= a_re * p[i].re - a_im * p[i].im;
          rh[i].im -= a_re * p[i].im + a_im * p[i].re;
        }
        // the even step after the last MR update reads e_o instead of rho
        const bool last_odd = k == nmr;
  #pragma unroll
        for (int i = 0; i < 6; i++) rho[(6 * h + i) * Vh + j] = last_odd ? eo[i] : rh[i];
        __syncthreads();
      }
    }
    } else {
    const int last = 2 * nmr + 1;
  #pragma unroll 1
    for (int step = 1; step <= last; step++) {
      const bool odd = (step & 1) == 0;
      Spinor<C> part;
      hops_inner(Vh, odd ? Vh + j : j, h, odd ? nbr_o : nbr_e, odd ? 0 : Vh, odd ? te : rho, Lt, part);
      cpx<C> hv[6], u[6], mu[6];
      exchange(xch, Vh, j, h, part, hv);
      // one clover multiply per step: A_oo rho (odd), A_ee^-1 D_eo rho (even),
      // A_ee^-1 (r_e - D_eo e_o) (last)
  #pragma unroll
      for (int i = 0; i < 6; i++)
        u[i] = odd ? rh[i] : (step == last ? cpx<C>{r_e[i].re - hv[i].re, r_e[i].im - hv[i].im} : hv[i]);
      clover_of<STAGE>(odd ? Ao : Ai, tm + (odd ? 64 : 0), j, h, m);
      herm6_mv(m, u, mu);
      if (odd) {
        cpx<C> p[6];
        C pr_re = 0, pr_im = 0, pp = 0;
  #pragma unroll
        for (int i = 0; i < 6; i++) {
          p[i] = {mu[i].re - hv[i].re, mu[i].im - hv[i].im};
          pr_re += p[i].re * rh[i].re + p[i].im * rh[i].im;
          pr_im += p[i].re * rh[i].im - p[i].im * rh[i].re;
          pp += p[i].re * p[i].re + p[i].im * p[i].im;
        }
        block_sum3<SHAPE != 0 ? NT / 32 : 0>(pr_re, pr_im, pp, red);
        C a_re = 0, a_im = 0;
        if (pp > (C)0) {
          a_re = pr_re / pp;
          a_im = pr_im / pp;
        }
  #pragma unroll
        for (int i = 0; i < 6; i++) {
          eo[i].re += a_re * rh[i].re - a_im * rh[i].im;
          eo[i].im += a_re * rh[i].im + a_im * rh[i].re;
          rh[i].re -= a_re * p[i].re - a_im * p[i].im;
          rh[i].im -= a_re * p[i].im + a_im * p[i].re;
        }
        // the even half-step after the last MR update reads e_o instead of rho
        const bool last_odd = step == 2 * nmr;
  #pragma unroll
        for (int i = 0; i < 6; i++) rho[(6 * h + i) * Vh + j] = last_odd ? eo[i] : rh[i];
      } else if (step == last) {
  #pragma unroll
        for (int i = 0; i < 6; i++) ee[i] = mu[i];
      } else {
  #pragma unroll
        for (int i = 0; i < 6; i++) te[(6 * h + i) * Vh + j] = mu[i];
      }
      __syncthreads();
    }
    }

    // ---- x += e: gather both halves through shared memory, then half 0
    // writes the even site j and half 1 the odd site j (and, when asked,
    // e to the corrections field and the odd-site residual rho to the
    // residual field)
  #pragma unroll
    for (int i = 0; i < 6; i++) {
      te[(6 * h + i) * Vh + j] = ee[i];
      xch[(6 * h + i) * Vh + j] = eo[i];
      if (mode & SAP_WRITE_R) rho[(6 * h + i) * Vh + j] = rh[i];
    }
    __syncthreads();
    {
      const cpx<C> *src = h ? xch : te;
      const int s = h ? Vh + j : j;
      Spinor<C> xs, e;
      vec_load(src, Vh, j, e);
      if ((mode & SAP_WRITE_E) && !flux) store_spinor<S, C>(ax.e[r], g, b, s, e);
      if ((mode & SAP_WRITE_R) && h) {
        Spinor<C> rs;
        vec_load(rho, Vh, j, rs);
        store_spinor<S, C>(ax.r[r], g, b, s, rs);
      }
      if (self_zero) {
        xs = e;
      } else {
        load_spinor<S, C>(xf, g, b, s, xs);
  #pragma unroll
        for (int i = 0; i < 12; i++) {
          xs.c[i].re += e.c[i].re;
          xs.c[i].im += e.c[i].im;
        }
      }
      store_spinor<S, C>(xf, g, b, s, xs);
    }
    if constexpr (sizeof(C) == 4)
      if ((mode & SAP_WRITE_E) && flux) flux_produce<S, C, P>(g, b, se.bc, Lt, te, xch, ax.e[r]);
    __syncthreads();   // shared vectors are reused by the next right-hand side
  }
  if (quit) break;
  }  // work items
  if constexpr (STAGE == 3) {
    // every thread's TMEM reads are complete; the allocating warp frees
    tmem_sync();
    if (threadIdx.x < 32) tmem_dealloc<TCOLS>(*tmem_at);
  }
}

template <typename S, int STAGE, int MINB, int NT, int SHAPE, bool UNROLL = false, bool MULTI = false>
int sap_k(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp, const AuxPtrs *ax, int tile,
          bool persistent, cudaStream_t st) {
  if (nl > 1 && !MULTI) {
    set_error("sap: this launch variant covers one lattice");
    return DD_EINVAL;
  }
  const Geom &g = L[0].g;   // every lattice of the launch has this block shape
  size_t smem = SapSmem<S>::bytes(g, STAGE);
  auto kern = k_sap_phase<S, STAGE, MINB, NT, SHAPE, UNROLL, MULTI>;
  // raise the kernel's dynamic shared-memory limit once (never during a capture)
  static std::mutex mu;
  static int raised = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (raised < (int)smem) {
      DD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
      raised = 227 * 1024;
    }
  }
  SapGroups G{};
  G.n = nl;
  int nitems = 0;
  for (int k = 0, rhs0 = 0; k < nl; k++) {
    G.grp[k] = SapGroup{L[k].g, L[k].f.links_full, L[k].f.clov, L[k].f.cinv, rhs0, L[k].nrhs, nitems};
    nitems += L[k].g.nblocks / 2 * ((L[k].nrhs + tile - 1) / tile);
    rhs0 += L[k].nrhs;
  }
  G.nitems = nitems;
  int grid = nitems;
  if (persistent) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, g.Vb, smem);
    if (occ < 1) occ = 1;
    grid = std::min(nitems, sms * occ);
  }
  const AuxPtrs none{};
  for (int sw = 0; sw < p.sweeps; sw++)
    for (int colour = 0; colour < 2; colour++) {
      // with x = 0 on entry: the first phase sees x = 0 everywhere, the
      // second still has x = 0 on its own (colour-1) blocks
      int self_zero = (p.x_is_zero && sw == 0) ? 1 : 0;
      int halo_zero = (p.x_is_zero && sw == 0 && colour == 0) ? 1 : 0;
      int mode = 0;
      if (ax) {
        // a block's residual: b on its first solve when x = 0 there (minus the
        // neighbours' corrections from colour 0 when it is colour 1), the
        // stored residual from the second sweep on; from a given x the first
        // sweep forms b - D x. Corrections are read by the next phase,
        // residuals by the same colour in the next sweep.
        if (p.x_is_zero && sw == 0) mode = SAP_INCR | SAP_FROM_B | (colour ? SAP_HALO_E : 0);
        else if (sw > 0) mode = SAP_INCR | SAP_HALO_E;
        if (!(sw == p.sweeps - 1 && colour == 1)) mode |= SAP_WRITE_E;
        if (sw + 1 < p.sweeps) mode |= SAP_WRITE_R;
      }
      kern<<<grid, g.Vb, smem, st>>>(G, rp, ax ? *ax : none, colour, self_zero, halo_zero, mode, p.mr_steps, tile,
                                     sap_timeout_counter());
      DD_LAUNCHED();
    }
  return DD_OK;
}

// the kernel specialised for the lattice's block shape when there is one
template <typename S, int STAGE, int MINB, int NT = 256>
int sap_t(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp, const AuxPtrs *ax, int tile,
          bool persistent, cudaStream_t st) {
  constexpr int SH = NT == 256 ? 1 : 2;   // the shape this thread count fits
  if (shape_of(L[0].g) == SH)
    return nl > 1 ? sap_k<S, STAGE, MINB, NT, SH, false, true>(L, nl, p, rp, ax, tile, persistent, st)
                  : sap_k<S, STAGE, MINB, NT, SH>(L, nl, p, rp, ax, tile, persistent, st);
  if constexpr (STAGE == 3) {   // TMEM clover: specialised shapes only
    set_error("sap: the TMEM clover layout exists for the specialised block shapes only");
    return (int)DD_EINVAL;
  } else {
    return nl > 1 ? sap_k<S, STAGE, MINB, NT, 0, false, true>(L, nl, p, rp, ax, tile, persistent, st)
                  : sap_k<S, STAGE, MINB, NT, 0>(L, nl, p, rp, ax, tile, persistent, st);
  }
}
// the MR loop unrolled by parity (specialised shape only)
template <typename S, int STAGE, int MINB, int NT = 256>
int sap_u(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp, const AuxPtrs *ax, int tile,
          bool persistent, cudaStream_t st) {
  constexpr int SH = NT == 256 ? 1 : 2;
  if (shape_of(L[0].g) != SH) {
    set_error("sap: the unrolled MR loop exists for the specialised block shapes only");
    return DD_EINVAL;
  }
  return sap_k<S, STAGE, MINB, NT, SH, true>(L, nl, p, rp, ax, tile, persistent, st);
}

template <typename S> constexpr bool sixteen_bit() {
  return Store<S>::prec == DD_F16 || Store<S>::prec == DD_BF16 || Store<S>::prec == DD_F16N;
}

// Launch variants: tiles staged in shared memory with one CTA per SM; tiles
// staged with two CTAs per SM (fits when the storage is 16-bit); only the
// links staged, with two CTAs per SM (when the full staging does not fit
// twice); tiles read through L1/L2 with two CTAs per SM; for 16-bit storage
// on the 4^4 shape with one right-hand side, the two-CTA layouts again with
// the MR loop unrolled by parity; for 32- and 16-bit storage on the
// specialised shapes, the links staged and the clover blocks in TMEM.
// Variants that do not fit are skipped. With several right-hand sides a CTA also solves `tile` of them with one
// staging of its block's operator (rhs_tile; 0 lets the autotuner choose).
template <typename S>
int sap_variants(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp, const AuxPtrs *ax,
                 cudaStream_t st) {
  const Geom &g = L[0].g;
  const size_t limit = 227 * 1024, half = 113 * 1024;
  const bool stage1 = SapSmem<S>::bytes(g, 1) <= limit;
  const bool stage2 = SapSmem<S>::bytes(g, 1) <= half;
  const bool links2 = !stage2 && SapSmem<S>::bytes(g, 2) <= half;
  const bool nost2 = SapSmem<S>::bytes(g, 0) <= half;
  if (!stage1 && SapSmem<S>::bytes(g, 0) > limit) {
    set_error("sap: block of %d sites needs more shared memory than available", g.Vb);
    return DD_EINVAL;
  }
  // links staged and the clover blocks in TMEM (32- and 16-bit storage on
  // the specialised shapes)
  constexpr bool tmem_ok = Store<S>::prec != DD_F64;
  const int sh = shape_of(g);
  int layouts[8], nlay = 0;
  if (g.Vb > 256) {
    // 512-site blocks (e.g. 8 x 4^3): 512 threads, one CTA per SM
    layouts[nlay++] = stage1 ? 3 : 4;
    if (tmem_ok && sh == 2 && SapSmem<S>::bytes(g, 3) <= limit) layouts[nlay++] = 9;
  } else {
    if (stage1) layouts[nlay++] = 0;
    if (stage2) layouts[nlay++] = 1;
    if (links2) layouts[nlay++] = 5;
    if (nost2 || !stage1) layouts[nlay++] = 2;
    // 16-bit storage on the 4^4 shape with one right-hand side: the two-CTA
    // layouts also with the MR loop unrolled by parity (measured faster
    // there, slower in multi-source tiles and for FP32)
    if (sixteen_bit<S>() && shape_of(g) == 1 && rp.n == 1) {
      if (stage2) layouts[nlay++] = 6;
      if (nost2 || !stage1) layouts[nlay++] = 7;
    }
    if (tmem_ok && sh == 1 && SapSmem<S>::bytes(g, 3) <= half) layouts[nlay++] = 8;
  }
  int tiles[6], nt = 0;
  if (p.rhs_tile > 0) {
    tiles[nt++] = p.rhs_tile < rp.n ? p.rhs_tile : rp.n;
  } else {
    const int cand[5] = {1, 2, 4, 8, 12};
    for (int c : cand)
      if (c <= rp.n) tiles[nt++] = c;
  }
  // variant k: layout k % nlay, RHS tile (k / nlay) % nt, persistent grid if k >= nlay * nt
  auto run = [&](int k) {
    const int layout = layouts[k % nlay], tile = tiles[(k / nlay) % nt];
    const bool pers = k >= nlay * nt;
    switch (layout) {
      case 1: return sap_t<S, 1, 2>(L, nl, p, rp, ax, tile, pers, st);
      case 2: return sap_t<S, 0, 2>(L, nl, p, rp, ax, tile, pers, st);
      case 3: return sap_t<S, 1, 1, 512>(L, nl, p, rp, ax, tile, pers, st);
      case 4: return sap_t<S, 0, 1, 512>(L, nl, p, rp, ax, tile, pers, st);
      case 5: return sap_t<S, 2, 2>(L, nl, p, rp, ax, tile, pers, st);
      case 8:
      case 9:
        if constexpr (tmem_ok) {
          if (layout == 8) return sap_t<S, 3, 2>(L, nl, p, rp, ax, tile, pers, st);
          return sap_t<S, 3, 1, 512>(L, nl, p, rp, ax, tile, pers, st);
        }
        return (int)DD_EINVAL;
      case 6:
      case 7:
        if constexpr (sixteen_bit<S>()) {
          if (layout == 6) return sap_u<S, 1, 2>(L, nl, p, rp, ax, tile, pers, st);
          return sap_u<S, 0, 2>(L, nl, p, rp, ax, tile, pers, st);
        }
        return (int)DD_EINVAL;
      default: return sap_t<S, 1, 1>(L, nl, p, rp, ax, tile, pers, st);
    }
  };
  int k = 0;
  // the tuner's key: lattice, precision, right-hand-side count, smoother
  // parameters and boundary; a launch over several lattices is tuned once
  // per block shape, precision and total right-hand-side count (a served
  // stream meets ever new mixes of lattices, each would otherwise be tuned)
  std::string key;
  if (nl == 1) {
    key = tune_key("sap", g, L[0].f.prec, rp.n) + "|" + std::to_string(p.sweeps) + "," +
          std::to_string(p.mr_steps) + "," + std::to_string(p.rhs_tile) + "," + std::to_string(g.antiperiodic);
  } else {
    Geom gb = g;   // the block shape only
    for (int mu = 0; mu < 4; mu++) gb.L[mu] = 0;
    key = tune_key("sap-lattices", gb, L[0].f.prec, rp.n) + "|" + std::to_string(p.sweeps) + "," +
          std::to_string(p.mr_steps) + "," + std::to_string(p.rhs_tile);
  }
  // the graph cache's key adds every lattice's extents, boundary and right-hand sides
  std::string shape;
  for (int k = 0; k < nl; k++)
    shape += "|" + std::to_string(L[k].g.L[0]) + "," + std::to_string(L[k].g.L[1]) + "," +
             std::to_string(L[k].g.L[2]) + "," + std::to_string(L[k].g.L[3]) + "," + std::to_string(L[k].nrhs) + "," +
             std::to_string(L[k].g.antiperiodic);
  // a graph may only replay where a fresh capture records the same arguments:
  // every lattice's field pointers are part of its key
  std::string fields;
  for (int k = 0; k < nl; k++)
    fields += std::to_string((uintptr_t)L[k].f.links_full) + "," + std::to_string((uintptr_t)L[k].f.clov) + "," +
              std::to_string((uintptr_t)L[k].f.cinv) + ";";
  // x is pure output when x_is_zero, so trial runs leave the same result
  if (p.x_is_zero) {
    int rc = tuned_variant(key, 2 * nlay * nt, run, st, &k);
    if (rc) return rc;
  } else {
    int c = tune_lookup(key);
    k = c >= 0 ? c : 0;
  }
  return sap_launch_as_graph(key + shape + "|" + fields, k, 2 * p.sweeps, rp, ax, [&] { return run(k); }, st);
}

}  // namespace

}  // namespace dd
