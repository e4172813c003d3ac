// dd_solve_noalloc: a solve that allocates no memory at all.
//
// Some callers cannot allocate device memory at solve time: code running
// inside a host callback or a CUDA-graph-building tool that forbids
// cudaMalloc, embedded users that hand this library a fixed memory budget up
// front, or processes that must not fragment or grow the device heap while a
// time-critical loop runs. For them this file keeps the whole FGMRES
// workspace (Krylov basis, preconditioned vectors, temporaries and the
// reduction partials) in one file-scope device array of fixed size. Every GPU
// that loads the library holds that array until the process exits.
//
// The solve itself is the same SAP-preconditioned FGMRES as dd_solve for one
// right-hand side, built from the same kernels in the same order, so its
// result matches dd_solve's to rounding (in practice bit for bit).
//
// Rules of use:
//  * the array is shared by every call in the process: calls whose GPU work
//    overlaps (different streams or threads, or several devices' host threads
//    touching the same device) race on it and give wrong results;
//  * it keeps whatever the previous call left; this call clears what must
//    start at zero (the initial iterate when no initial guess is given) and
//    writes every other buffer before reading it;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current); make that first call
//    before any stream capture on the device. The address is kept for the
//    life of the process, so do not use this entry point on a device after
//    cudaDeviceReset in the same process;
//  * no launch-configuration tuning and no CUDA-graph capture happen inside
//    the call: each kernel runs in the variant the tuner has already chosen
//    for this lattice and precision (by an earlier dd_solve, dd_apply_D or
//    dd_sap_smooth in this process, or a DD_TUNE_CACHE file), or else in
//    its default variant, and the smoother's launches are enqueued one by
//    one on the caller's stream;
//  * the host side keeps its small arrays (the Hessenberg matrix of up to 64
//    columns and the rotations, about 72 KB) on the calling thread's stack.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>

#include "dd_solver.cuh"
#include "dd_tune.cuh"

namespace dd {
namespace {

static __device__ __align__(256) unsigned char g_scratch[DD_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(void **out) {
  int dev = 0;
  DD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("dd_solve_noalloc: device %d out of range", dev);
    return DD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DD_OK;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carve {
  char *base;
  size_t used = 0;
  template <typename T> T *take(size_t bytes) {
    T *p = (T *)(base + used);
    used += (bytes + 255) / 256 * 256;
    return p;
  }
};

using cd = std::complex<double>;
constexpr int MAXM = 64;

}  // namespace

size_t noalloc_bytes_needed(const Geom &g, int prec, int m, int nblk) {
  const int zprec = prec == DD_F64 ? DD_F64 : DD_F32;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t f64 = (size_t)g.V * 24 * 8, fz = (size_t)g.V * spinor_site_bytes(zprec), fp = (size_t)g.V * spinor_site_bytes(prec);
  return al(sizeof(double) * (size_t)nblk * 33) + al(sizeof(double) * 256) + al(sizeof(double) * 136) +
         al(sizeof(double) * 2 * MAXM) + (size_t)(m + 1) * al(f64) + (size_t)m * al(fz) + 4 * al(f64) + 4 * al(fp) +
         al(fz);
}

}  // namespace dd

using namespace dd;

extern "C" int dd_solve_noalloc(dd_op_t opp, const dd_solve_params *p, const double *b_dev, double *x_dev,
                                dd_solve_info *info, void *stream) {
  Op *op = (Op *)opp;
  if (!op || op->magic != 0x4f505231 || !b_dev || !x_dev) {
    set_error("dd_solve_noalloc: bad argument");
    return DD_EINVAL;
  }
  int rc = check_solve_params(p);
  if (rc) return rc;
  if (p->mg) {
    set_error("dd_solve_noalloc: the multigrid preconditioner needs workspace; use dd_solve");
    return DD_EINVAL;
  }
  const Geom &g = op->lat->g;
  const int m = p->restart;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  DD_CUDA(cudaGetDevice(&dev));
  DD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nblk = sms > 0 ? 4 * sms : 608;
  const size_t need = noalloc_bytes_needed(g, op->prec, m, nblk);
  if (need > (size_t)DD_NOALLOC_SCRATCH_BYTES) {
    set_error("dd_solve_noalloc: this lattice (%lld sites) with restart %d needs %zu bytes of scratch, more than "
              "the built-in %zu; use dd_solve", (long long)g.V, m, need, (size_t)DD_NOALLOC_SCRATCH_BYTES);
    return DD_EINVAL;
  }
  void *base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  // no tuning trial launches and no graph capture below (see the header)
  DirectLaunch direct;

  // carve the workspace
  const int zprec = op->prec == DD_F64 ? DD_F64 : DD_F32;
  const bool df = zprec == DD_F32 && !p->outer_f64;
  const size_t n = (size_t)g.V * 12, f64 = (size_t)g.V * 24 * 8;
  const size_t fz = (size_t)g.V * spinor_site_bytes(zprec), fp = (size_t)g.V * spinor_site_bytes(op->prec);
  const size_t fz_al = (fz + 255) / 256 * 256, f64_al = (f64 + 255) / 256 * 256;
  Carve cv{(char *)base};
  Blas bl;
  bl.nblk = nblk;
  bl.partial = cv.take<double>(sizeof(double) * (size_t)nblk * 33);
  bl.result = cv.take<double>(sizeof(double) * 256);
  double *hd = cv.take<double>(sizeof(double) * 136);
  double *yd = cv.take<double>(sizeof(double) * 2 * MAXM);
  double *Vb = cv.take<double>((size_t)(m + 1) * f64_al);
  char *Z = cv.take<char>((size_t)m * fz_al);
  double *x = cv.take<double>(f64), *b = cv.take<double>(f64), *w = cv.take<double>(f64);
  double *canon = cv.take<double>(f64);
  void *tin = cv.take<char>(fp), *tout = cv.take<char>(fp), *zt = cv.take<char>(fz);
  AuxPtrs ax{};   // the smoother's work fields (corrections, block residuals)
  ax.e[0] = cv.take<char>(fp);
  ax.r[0] = cv.take<char>(fp);
  const size_t vstride = f64_al / 16;   // complex entries between basis vectors

  // the Blas object borrows scratch; detach it before it goes out of scope
  struct Detach {
    Blas &b;
    ~Detach() { b.partial = b.result = nullptr; }
  } detach{bl};

  const double sigma = std::sqrt(24.0 * (double)g.V);
  auto t0 = std::chrono::steady_clock::now();
  double hh[136];
  cd H[(MAXM + 1) * MAXM], gv[MAXM + 1], sn[MAXM], y[MAXM];
  double cs[MAXM];
  int its = 0, cycles = 0, status = DD_ENOTCONV;
  double bnorm = -1, rel = 1, est = 1;

  // b, x0 into the FP64 field layout
  DD_CUDA(cudaMemcpyAsync(canon, b_dev, f64, cudaMemcpyDeviceToDevice, st));
  if ((rc = launch_pack(g, DD_F64, canon, b, 1, 1.0, st))) return rc;
  if (p->use_x0) {
    DD_CUDA(cudaMemcpyAsync(canon, x_dev, f64, cudaMemcpyDeviceToDevice, st));
    if ((rc = launch_pack(g, DD_F64, canon, x, 1, 1.0, st))) return rc;
  } else {
    DD_CUDA(cudaMemsetAsync(x, 0, f64, st));
  }
  const OpFields &fz_ops = zprec == DD_F64 ? op->f64 : op->f32;
  bool x_zero = !p->use_x0;   // first cycle from x = 0: D x = 0, no Dslash
  for (;;) {
    // true residual r = b - D x (FP64) in w
    if (x_zero) {
      DD_CUDA(cudaMemsetAsync(w, 0, f64, st));
      x_zero = false;
    } else if (df) {   // double-float Dslash on the pre-split fields, as dd_solve
      if ((rc = launch_split_pairs(x, canon, n, st))) return rc;
      if ((rc = launch_dirac_df(g, op->fdf, contiguous(canon, w, 1, f64), st))) return rc;
    } else if ((rc = launch_dirac(g, op->f64, x, w, 1, st))) {
      return rc;
    }
    if ((rc = bl.xmy(b, w, n, st))) return rc;
    if ((rc = bl.norm2(w, n, hd + 132, st))) return rc;
    if (bnorm < 0 && (rc = bl.norm2(b, n, hd + 133, st))) return rc;
    DD_CUDA(cudaMemcpyAsync(hh, hd, sizeof hh, cudaMemcpyDeviceToHost, st));
    DD_CUDA(cudaStreamSynchronize(st));
    if (bnorm < 0) bnorm = std::sqrt(hh[133]);
    const double beta = std::sqrt(hh[132]);
    if (bnorm == 0) {
      DD_CUDA(cudaMemsetAsync(x, 0, f64, st));
      rel = est = 0;
      status = DD_OK;
      break;
    }
    rel = beta / bnorm;
    if (!std::isfinite(rel)) break;
    if (rel <= p->tol) {
      est = rel;
      status = DD_OK;
      break;
    }
    if (its >= p->max_iter) break;
    cycles++;
    for (int i = 0; i <= m; i++) gv[i] = 0;
    gv[0] = beta;
    const double target = std::max(p->tol * bnorm, p->inner_reduction * beta);
    if (df) rc = bl.f64_to_df((float *)Vb, w, 1.0 / beta, n, st);
    else rc = bl.scale(Vb, w, 1.0 / beta, n, st);
    if (rc) return rc;
    int j = 0;
    for (;; j++) {
      double *vj = Vb + 2 * vstride * j;
      char *zj = Z + (size_t)j * fz_al;
      if (df) rc = bl.df_to_field(g, (const float *)vj, op->prec, tin, sigma, st);
      else rc = launch_convert_field(g, DD_F64, vj, op->prec, tin, 1, sigma, st);
      if (rc) return rc;
      dd_sap_params sp = p->sap;
      sp.x_is_zero = 1;
      // z_j = SAP(sigma v_j), kept scaled by sigma as in dd_solve (H and y carry the factor)
      if (op->prec == zprec) {
        if ((rc = launch_sap(g, op->fp, sp, contiguous(tin, zj, 1, fp), st, &ax))) return rc;
      } else {
        if ((rc = launch_sap(g, op->fp, sp, contiguous(tin, tout, 1, fp), st, &ax))) return rc;
        if ((rc = launch_convert_field(g, op->prec, tout, zprec, zj, 1, 1.0, st))) return rc;
      }
      if ((rc = launch_dirac(g, fz_ops, zj, zprec == DD_F64 ? (void *)w : zt, 1, st))) return rc;
      if (zprec != DD_F64) {
        rc = df ? bl.field_to_df(g, DD_F32, zt, (float *)w, st) : launch_convert_field(g, DD_F32, zt, DD_F64, w, 1, 1.0, st);
        if (rc) return rc;
      }
      const int kk = j + 1;
      auto mdot = [&](double *wn2) {
        return df ? bl.df_mdot((const float *)Vb, vstride, kk, (const float *)w, n, hd, wn2, st)
                  : bl.mdot(Vb, vstride, kk, w, n, hd, wn2, st);
      };
      auto maxpy = [&]() {
        return df ? bl.df_maxpy_norm((const float *)Vb, vstride, kk, hd, (float *)w, n, hd + 131, st)
                  : bl.maxpy_norm(Vb, vstride, kk, hd, w, n, hd + 131, st);
      };
      if ((rc = mdot(hd + 130)) || (rc = maxpy())) return rc;
      DD_CUDA(cudaMemcpyAsync(hh, hd, sizeof hh, cudaMemcpyDeviceToHost, st));
      DD_CUDA(cudaStreamSynchronize(st));
      cd hcol[MAXM];
      for (int q = 0; q < kk; q++) hcol[q] = cd(hh[2 * q], hh[2 * q + 1]);
      if (hh[131] < REORTH2 * hh[130]) {
        if ((rc = mdot(nullptr)) || (rc = maxpy())) return rc;
        DD_CUDA(cudaMemcpyAsync(hh, hd, sizeof hh, cudaMemcpyDeviceToHost, st));
        DD_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < kk; q++) hcol[q] += cd(hh[2 * q], hh[2 * q + 1]);
      }
      its++;
      const double hn = std::sqrt(std::max(hh[131], 0.0));
      for (int q = 0; q < kk; q++) H[q * m + j] = hcol[q];
      if (hn > 0) {
        double *vn = Vb + 2 * vstride * (j + 1);
        if (df) rc = bl.df_scale((float *)vn, (const float *)w, 1.0 / hn, n, st);
        else rc = bl.scale(vn, w, 1.0 / hn, n, st);
        if (rc) return rc;
      }
      for (int q = 0; q < j; q++) {
        cd a = H[q * m + j], c2 = H[(q + 1) * m + j];
        H[q * m + j] = cs[q] * a + sn[q] * c2;
        H[(q + 1) * m + j] = -std::conj(sn[q]) * a + cs[q] * c2;
      }
      cd a = H[j * m + j];
      const double rr = std::sqrt(std::norm(a) + hn * hn);
      if (std::abs(a) == 0) {
        cs[j] = 0;
        sn[j] = 1;
      } else {
        cs[j] = std::abs(a) / rr;
        sn[j] = (a / std::abs(a)) * hn / rr;
      }
      H[j * m + j] = cs[j] * a + sn[j] * hn;
      gv[j + 1] = -std::conj(sn[j]) * gv[j];
      gv[j] = cs[j] * gv[j];
      est = std::abs(gv[j + 1]) / bnorm;
      if (std::abs(gv[j + 1]) <= target || j + 1 == m || its >= p->max_iter || hn == 0) break;
    }
    // y = R^-1 g ; x += Z y
    const int k = j + 1;
    for (int i = k - 1; i >= 0; i--) {
      cd t = gv[i];
      for (int l = i + 1; l < k; l++) t -= H[i * m + l] * y[l];
      y[i] = t / H[i * m + i];
    }
    double yh[2 * MAXM];
    for (int i = 0; i < k; i++) {
      yh[2 * i] = y[i].real();
      yh[2 * i + 1] = y[i].imag();
    }
    DD_CUDA(cudaMemcpyAsync(yd, yh, sizeof(double) * 2 * k, cudaMemcpyHostToDevice, st));
    if ((rc = bl.update_x(g, x, zprec, Z, fz_al, k, yd, st))) return rc;
  }
  if ((rc = launch_unpack(g, DD_F64, x, canon, 1, 1.0, st))) return rc;
  DD_CUDA(cudaMemcpyAsync(x_dev, canon, f64, cudaMemcpyDeviceToDevice, st));
  DD_CUDA(cudaStreamSynchronize(st));
  if (info) {
    info->status = status;
    info->iterations = its;
    info->cycles = cycles;
    info->true_rel_residual = rel;
    info->est_rel_residual = est;
    info->ms_sap = info->ms_dirac = info->ms_orth = 0;
    info->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status != DD_OK) {
    set_error("dd_solve_noalloc: max_iter reached before the target residual");
    return DD_ENOTCONV;
  }
  return DD_OK;
}
