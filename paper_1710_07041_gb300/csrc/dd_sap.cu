// Schwarz alternating procedure (Sec. 3.1, Table 2 "Schwarz method") with the
// block solve by minimal-residual steps (Sec. 3.1, Table 1 "MR inversion
// within a domain"). Red-black multiplicative Schwarz: per sweep, all blocks
// of colour 0 and then all blocks of colour 1 are solved, each from the
// current global residual, and the block correction is added to x.
//
// One CTA per block (x one right-hand side). Per phase the CTA
//   1. stages the block's links, odd-site clover A_oo and even-site inverse
//      A_ee^-1 into shared memory with bulk (TMA) copies (overlapping step 2;
//      in one layout the clover blocks go to tensor memory instead, each
//      thread's two blocks into its own TMEM lane),
//   2. forms its residual: r = b - D x on its sites (neighbour x read from
//      the other colour's blocks in HBM; skipped when x = 0), or, given work
//      fields, incrementally: after its own solve a block's residual is zero
//      on even sites and the MR residual rho on odd ones, and until its next
//      phase only the neighbouring blocks' corrections e change x, so
//      r = (stored residual, or b on the first solve from x = 0) minus the
//      hops of e across the block faces; each phase stores its rho and, as
//      face flux, the hops of its e into the neighbouring blocks' face sites
//      (computed from the staged links and e in shared memory; the receiver
//      reads its flux contiguously) for the next phases (DD_SAP_INCR=0
//      turns this off),
//   3. Schur right-hand side  bhat = r_o - D_oe A_ee^-1 r_e,
//   4. n_MR steps on Dhat = A_oo - D_oe A_ee^-1 D_eo from e_o = 0:
//        p = Dhat rho, alpha = <p,rho>/<p,p>, e_o += alpha rho, rho -= alpha p,
//   5. reconstructs e_e = A_ee^-1 (r_e - D_eo e_o) and writes x += e.
// All MR vectors stay in shared memory for the whole block solve. Threads:
// 2 per even/odd site pair; thread half h owns spin components {2h, 2h+1}
// (chirality block h of the clover) and evaluates the hops in directions
// {2h, 2h+1}; the two halves exchange partial hop sums through shared memory.
// With Vh = block sites / 2 a multiple of 32, h is warp-uniform, so the
// per-direction code never diverges inside a warp.
// This file holds the host side (variant dispatch per storage precision, the
// graph cache, the wait counter); the kernel templates are in
// dd_sap_kernels.cuh and instantiated per precision in dd_sap_<prec>.cu.
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "dd_sap_kernels.cuh"

namespace dd {

// Number of bounded device waits that expired (read and cleared by
// dd_device_status).
__device__ unsigned g_wait_timeouts = 0;

int device_wait_status() {
  int rc = cuda_fail(cudaDeviceSynchronize(), "device status");
  if (rc) return rc;
  if (const unsigned nb = bounds_errors_all()) {   // checked builds only
    set_error("%u out-of-range indices caught by the checked build", nb);
    return DD_ECUDA;
  }
  unsigned n = 0, zero = 0;
  if ((rc = cuda_fail(cudaMemcpyFromSymbol(&n, g_wait_timeouts, sizeof(n)), "device status"))) return rc;
  if (n) {
    if ((rc = cuda_fail(cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(zero)), "device status"))) return rc;
    set_error("%u bounded device wait(s) expired", n);
    return DD_ETIMEOUT;
  }
  return DD_OK;
}


// device address of g_wait_timeouts on the current device (cached per device)
unsigned *sap_timeout_counter() {
  static std::mutex mu;
  static std::map<int, unsigned *> addr;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) return it->second;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_wait_timeouts) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  addr[dev] = (unsigned *)p;
  return (unsigned *)p;
}

int sap_run_f64(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                const AuxPtrs *ax, cudaStream_t st);
int sap_run_f32(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                const AuxPtrs *ax, cudaStream_t st);
int sap_run_f16(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                const AuxPtrs *ax, cudaStream_t st);
int sap_run_f16n(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                 const AuxPtrs *ax, cudaStream_t st);
int sap_run_bf16(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp,
                const AuxPtrs *ax, cudaStream_t st);

namespace {
// Self-test of the staging handshake: one 16-byte bulk copy tracked by an
// mbarrier; with `expire` the barrier is told to expect 16 more bytes than
// are copied, so its phase never completes and the bounded wait must expire.
// result: 0 copy landed, 1 wait expired, 2 copy landed with wrong data.
__global__ void k_wait_selftest(const uint4 *src, int expire, int *result, unsigned *timeouts) {
  __shared__ __align__(16) uint4 buf;
  __shared__ __align__(8) uint64_t mbar;
  const unsigned m = smem_u32(&mbar);
  if (threadIdx.x == 0) mbar_init(&mbar);
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_proxy_async();
    mbar_arrive_expect(&mbar, expire ? 32u : 16u);
    bulk_g2s(&buf, src, 16u, &mbar);
  }
  const bool ok = mbar_wait(m, 0);
  if (__syncthreads_or(!ok)) {
    wait_expired(timeouts, m, 0);
    if (threadIdx.x == 0) *result = 1;
    return;
  }
  if (threadIdx.x == 0) *result = (buf.x == src->x && buf.w == src->w) ? 0 : 2;
}

}  // namespace

// The 2 x sweeps phase launches of one smoother application are captured once
// into a CUDA graph per (operator, parameters, variant, field pointers) and
// replayed afterwards: one launch per application instead of 2 x sweeps.
// When the caller's stream is itself being captured the launches go into the
// caller's graph directly. DD_SAP_GRAPHS=0 disables the graphs, and so does
// a DirectLaunch scope on the calling thread (dd_solve_noalloc).
// An instantiated graph, destroyed when its last holder lets go: a thread
// that looked one up keeps it alive through its launch even if another thread
// flushes the cache meanwhile (a destroyed graph that is still running on the
// device is freed by the driver once it completes).
struct GraphExec {
  cudaGraphExec_t exec = nullptr;
  ~GraphExec() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};
struct GraphCache {
  std::mutex mu;
  std::map<std::string, std::shared_ptr<GraphExec>> execs;
};
// never destroyed: no CUDA call runs at process exit
static GraphCache &g_graphs = *new GraphCache;

int sap_launch_as_graph(const std::string &key, int variant, int nkernels, const RhsPtrs &rp, const AuxPtrs *ax,
                        const std::function<int()> &enqueue, cudaStream_t st) {
  const char *env = getenv("DD_SAP_GRAPHS");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if ((env && env[0] == '0') || cap != cudaStreamCaptureStatusNone || st == 0 || direct_launch()) return enqueue();
  // every pointer baked into the captured launches is part of the key (a
  // graph may only be replayed where a fresh capture would record the same
  // arguments; the caller's key holds the geometry and the operator fields)
  std::string k = key + "|v" + std::to_string(variant);
  for (int i = 0; i < rp.n; i++) {
    k += "|" + std::to_string((uintptr_t)rp.in[i]) + ":" + std::to_string((uintptr_t)rp.out[i]);
    if (ax) k += ":" + std::to_string((uintptr_t)ax->e[i]) + ":" + std::to_string((uintptr_t)ax->r[i]);
  }
  std::shared_ptr<GraphExec> held;
  {
    std::lock_guard<std::mutex> lk(g_graphs.mu);
    auto it = g_graphs.execs.find(k);
    if (it != g_graphs.execs.end()) held = it->second;
  }
  if (!held) {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    DD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue();
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "sap graph capture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "sap graph instantiate");
    held = std::make_shared<GraphExec>();
    held->exec = exec;
    std::lock_guard<std::mutex> lk(g_graphs.mu);
    if (g_graphs.execs.size() >= 256) g_graphs.execs.clear();   // bounded cache: start over when full
    // (another thread may have stored the same key meanwhile: this one's
    // graph is then launched once and freed)
    g_graphs.execs.emplace(k, held);
  } else {
    count_launches(nkernels);
  }
  return cuda_fail(cudaGraphLaunch(held->exec, st), "sap graph launch");
}


int wait_selftest(int expire) {
  uint4 *src = nullptr;
  int *res = nullptr;
  DD_CUDA(cudaMalloc(&src, sizeof(uint4) + sizeof(int)));
  res = (int *)(src + 1);
  const uint4 pat = make_uint4(0x01234567u, 0x89abcdefu, 0x0f1e2d3cu, 0x4b5a6978u);
  int got = -1, rc = cuda_fail(cudaMemcpy(src, &pat, sizeof(pat), cudaMemcpyHostToDevice), "wait selftest");
  if (rc == DD_OK) {
    unsigned *cnt = sap_timeout_counter();
    if (!cnt) return cuda_fail(cudaErrorInvalidSymbol, "wait selftest");
    k_wait_selftest<<<1, 32>>>(src, expire, res, cnt);
    rc = launched("k_wait_selftest");
  }
  if (rc == DD_OK) rc = cuda_fail(cudaMemcpy(&got, res, sizeof(int), cudaMemcpyDeviceToHost), "wait selftest");
  cudaFree(src);
  if (rc) return rc;
  if (got != (expire ? 1 : 0)) {
    set_error("wait selftest: result %d (expected %d)", got, expire ? 1 : 0);
    return DD_ECUDA;
  }
  return DD_OK;
}

size_t sap_smem_bytes(const Geom &g, int prec, bool stage) {
  switch (prec) {
    case DD_F64: return SapSmem<double>::bytes(g, stage ? 1 : 0);
    case DD_F32: return SapSmem<float>::bytes(g, stage ? 1 : 0);
    case DD_F16: return SapSmem<__half>::bytes(g, stage ? 1 : 0);
    case DD_F16N: return SapSmem<hn16>::bytes(g, stage ? 1 : 0);
    default: return SapSmem<__nv_bfloat16>::bytes(g, stage ? 1 : 0);
  }
}

int launch_sap(const Geom &g, const OpFields &f, const dd_sap_params &p, const void *b, void *x, int nrhs,
               cudaStream_t st, void *aux_base) {
  const size_t fb = (size_t)g.V * spinor_site_bytes(f.prec);
  for (int r0 = 0; r0 < nrhs; r0 += MAX_RHS) {
    int n = nrhs - r0 < MAX_RHS ? nrhs - r0 : MAX_RHS;
    AuxPtrs ax{};
    for (int i = 0; aux_base && i < n; i++) {
      ax.e[i] = (char *)aux_base + (size_t)(r0 + i) * fb;
      ax.r[i] = (char *)aux_base + (size_t)(nrhs + r0 + i) * fb;
    }
    int rc = launch_sap(g, f, p, contiguous((const char *)b + r0 * fb, (char *)x + r0 * fb, n, fb), st,
                        aux_base ? &ax : nullptr);
    if (rc) return rc;
  }
  return DD_OK;
}

int launch_sap(const Geom &g, const OpFields &f, const dd_sap_params &p, const RhsPtrs &rp, cudaStream_t st,
               const AuxPtrs *ax) {
  const SapLattice L{g, f, rp.n};
  return launch_sap_lattices(&L, 1, p, rp, st, ax);
}

int launch_sap_lattices(const SapLattice *L, int nl, const dd_sap_params &p, const RhsPtrs &rp, cudaStream_t st,
                        const AuxPtrs *ax) {
  NvtxRange range("dd:sap");
  if (nl < 1 || nl > MAX_SAP_GROUPS) {
    set_error("sap: 1..%d lattices per launch", MAX_SAP_GROUPS);
    return DD_EINVAL;
  }
  int total = 0;
  for (int k = 0; k < nl; k++) {
    total += L[k].nrhs;
    bool same = L[k].f.prec == L[0].f.prec && L[k].nrhs >= 1;
    for (int mu = 0; mu < 4; mu++) same = same && L[k].g.bd[mu] == L[0].g.bd[mu];
    if (!same) {
      set_error("sap: the lattices of one launch need the same block shape and precision, and right-hand sides");
      return DD_EINVAL;
    }
  }
  if (total != rp.n) {
    set_error("sap: %d right-hand sides given for %d in the lattices", rp.n, total);
    return DD_EINVAL;
  }
  const Geom &g = L[0].g;
  const OpFields &f = L[0].f;
  // DD_SAP_INCR=0: every phase forms r = b - D x from x (the incremental
  // colour residual is off even where work fields are given)
  static const bool incr_off = [] {
    const char *e = getenv("DD_SAP_INCR");
    return e && e[0] == '0';
  }();
  if (incr_off) ax = nullptr;
  if (rp.n < 1 || rp.n > MAX_RHS) {
    set_error("sap: 1..%d right-hand sides per launch", MAX_RHS);
    return DD_EINVAL;
  }
  if (g.Vb > 512) {
    set_error("sap: blocks of more than 512 sites are not supported (got %d)", g.Vb);
    return DD_EINVAL;
  }
  if (!sap_timeout_counter()) {   // resolved here, before any graph capture of the launches
    set_error("sap: wait counter not available");
    return DD_ECUDA;
  }
  switch (f.prec) {
    case DD_F64: return sap_run_f64(L, nl, p, rp, ax, st);
    case DD_F32: return sap_run_f32(L, nl, p, rp, ax, st);
    case DD_F16: return sap_run_f16(L, nl, p, rp, ax, st);
    case DD_BF16: return sap_run_bf16(L, nl, p, rp, ax, st);
    case DD_F16N: return sap_run_f16n(L, nl, p, rp, ax, st);
  }
  set_error("sap: bad precision %d", f.prec);
  return DD_EINVAL;
}

}  // namespace dd
