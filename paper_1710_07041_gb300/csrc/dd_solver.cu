// Outer solver: FGMRES(m) right-preconditioned by the Schwarz method
// (Saad 1993). The paper calls DD-alpha-AMG for the Dirac equation (Sec. 1)
// with SAP as its fine-grid smoother (Sec. 3.1); this library runs the
// SAP-preconditioned fine-grid Krylov solve, with mixed precision in the
// spirit of Sec. 3.1's half-precision storage: the smoother works in the
// operator's storage precision, while the Arnoldi orthogonalisation, the
// least-squares update and the true residual are FP64. Preconditioned
// vectors z_j are kept in FP32 (FP64 for an FP64 operator), and the Arnoldi
// product D z_j uses the operator in that same precision, so D Z = V H holds
// to that precision; every cycle ends with the FP64 true residual, so the
// restarts act as iterative refinement.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "dd_blas.cuh"
#include "dd_solver.cuh"

namespace dd {

using cd = std::complex<double>;

SolveWork::~SolveWork() { release(); }

void SolveWork::release() {
  void *ptrs[] = {Vb, Z, w, r, x, b, tmp, tin, tout, zt, canon, hdev, ydev};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  Vb = nullptr; Z = nullptr; w = r = x = b = tmp = nullptr; tin = tout = zt = nullptr; canon = nullptr;
  hdev = ydev = nullptr;
  for (auto &e : ev)
    if (e) { cudaEventDestroy(e); e = nullptr; }
  bytes = 0;
}

size_t SolveWork::bytes_needed(const Geom &g, int prec, int m) {
  size_t f64 = (size_t)g.V * 24 * 8;
  int zprec = prec == DD_F64 ? DD_F64 : DD_F32;
  size_t fz = (size_t)g.V * 24 * real_bytes(zprec), fp = (size_t)g.V * 24 * real_bytes(prec);
  return (size_t)(m + 1) * f64 + (size_t)m * fz + 6 * f64 + 2 * fp + fz + (1 << 16);
}

int SolveWork::ensure(const Geom &g, int prec_, int m_) {
  if (Vb && m_ <= m && prec_ == prec && g.V == V) return DD_OK;
  release();
  prec = prec_;
  m = m_;
  V = g.V;
  zprec = prec == DD_F64 ? DD_F64 : DD_F32;
  size_t f64 = (size_t)g.V * 24 * 8;
  zbytes = (size_t)g.V * 24 * real_bytes(zprec);
  pbytes = (size_t)g.V * 24 * real_bytes(prec);
  bool ok = cudaMalloc((void **)&Vb, (size_t)(m + 1) * f64) == cudaSuccess &&
            cudaMalloc(&Z, (size_t)m * zbytes) == cudaSuccess && cudaMalloc((void **)&w, f64) == cudaSuccess &&
            cudaMalloc((void **)&r, f64) == cudaSuccess && cudaMalloc((void **)&x, f64) == cudaSuccess &&
            cudaMalloc((void **)&b, f64) == cudaSuccess && cudaMalloc((void **)&tmp, f64) == cudaSuccess &&
            cudaMalloc((void **)&canon, f64) == cudaSuccess && cudaMalloc(&tin, pbytes) == cudaSuccess &&
            cudaMalloc(&tout, pbytes) == cudaSuccess && cudaMalloc(&zt, zbytes) == cudaSuccess &&
            cudaMalloc((void **)&hdev, sizeof(double) * 4 * 80) == cudaSuccess &&
            cudaMalloc((void **)&ydev, sizeof(double) * 2 * 80) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release();
    set_error("dd_solve: out of device memory for the FGMRES(%d) workspace", m_);
    return DD_ENOMEM;
  }
  for (auto &e : ev) DD_CUDA(cudaEventCreate(&e));
  if (!blas.partial) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int rc = blas.init(sms);
    if (rc) return rc;
  }
  bytes = bytes_needed(g, prec, m);
  return DD_OK;
}

namespace {

double host_norm2(Blas &bl, const double *v, size_t n, cudaStream_t st, int *rc) {
  *rc = bl.norm2(v, n, bl.result + 200, st);
  if (*rc) return 0;
  *rc = cuda_fail(cudaMemcpyAsync(bl.hpin, bl.result + 200, sizeof(double), cudaMemcpyDeviceToHost, st), "norm");
  if (!*rc) *rc = cuda_fail(cudaStreamSynchronize(st), "norm sync");
  return bl.hpin[0];
}

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float t = 0;
  cudaEventElapsedTime(&t, a, b);
  return t;
}

}  // namespace

// One right-hand side: W.b holds b (FP64 field), W.x the initial guess.
int fgmres_one(const Op *op, const dd_solve_params &p, SolveWork &W, dd_solve_info &info, cudaStream_t st,
               const volatile int *cancel) {
  const Geom &g = op->lat->g;
  const size_t n = (size_t)g.V * 12;  // complex entries of one field
  const int m = p.restart;
  const double sigma = std::sqrt(24.0 * (double)g.V);  // unit-norm vector -> unit RMS entries
  Blas &bl = W.blas;
  int rc = 0;
  auto t0 = std::chrono::steady_clock::now();
  double ms_sap = 0, ms_dirac = 0, ms_orth = 0;

  double bnorm = std::sqrt(host_norm2(bl, W.b, n, st, &rc));
  if (rc) return rc;
  info.iterations = info.cycles = 0;
  if (bnorm == 0) {
    DD_CUDA(cudaMemsetAsync(W.x, 0, n * 16, st));
    DD_CUDA(cudaStreamSynchronize(st));
    info.status = DD_OK;
    info.true_rel_residual = info.est_rel_residual = 0;
    return DD_OK;
  }
  std::vector<cd> H((size_t)(m + 1) * m), gv(m + 1), sn(m), y(m);
  std::vector<double> cs(m);
  int its = 0;
  double rel = 1, est = 1;
  int status = DD_ENOTCONV;
  for (;;) {
    // true residual r = b - D x (FP64)
    cudaEventRecord(W.ev[0], st);
    if ((rc = launch_dirac(g, op->f64, W.x, W.r, 1, st))) return rc;
    if ((rc = bl.xmy(W.b, W.r, n, st))) return rc;
    cudaEventRecord(W.ev[1], st);
    double beta = std::sqrt(host_norm2(bl, W.r, n, st, &rc));
    if (rc) return rc;
    ms_dirac += ev_ms(W.ev[0], W.ev[1]);
    rel = beta / bnorm;
    if (!std::isfinite(rel)) {
      set_error("dd_solve: residual is not finite");
      status = DD_ENOTCONV;
      break;
    }
    if (rel <= p.tol) { status = DD_OK; est = rel; break; }
    if (its >= p.max_iter) { status = DD_ENOTCONV; break; }
    if (cancel && *cancel) { status = DD_ECANCELLED; break; }
    info.cycles++;
    if ((rc = bl.scale(W.Vb, W.r, 1.0 / beta, n, st))) return rc;
    std::fill(gv.begin(), gv.end(), cd(0));
    gv[0] = beta;
    const double target = std::max(p.tol * bnorm, p.inner_reduction * beta);
    int k = 0;
    for (int j = 0; j < m && its < p.max_iter; j++) {
      double *vj = W.Vb + 2 * n * j;
      char *zj = (char *)W.Z + (size_t)j * W.zbytes;
      // z_j = SAP(v_j) in the smoother's precision, kept in zprec
      cudaEventRecord(W.ev[0], st);
      if ((rc = launch_convert_field(g, DD_F64, vj, op->prec, W.tin, 1, sigma, st))) return rc;
      dd_sap_params sp = p.sap;
      sp.x_is_zero = 1;
      if ((rc = launch_sap(g, op->fp, sp, W.tin, W.tout, 1, st))) return rc;
      if ((rc = launch_convert_field(g, op->prec, W.tout, W.zprec, zj, 1, 1.0 / sigma, st))) return rc;
      cudaEventRecord(W.ev[1], st);
      // w = D z_j
      if (W.zprec == DD_F64) {
        if ((rc = launch_dirac(g, op->f64, zj, W.w, 1, st))) return rc;
      } else {
        if ((rc = launch_dirac(g, op->f32, zj, W.zt, 1, st))) return rc;
        if ((rc = launch_convert_field(g, DD_F32, W.zt, DD_F64, W.w, 1, 1.0, st))) return rc;
      }
      cudaEventRecord(W.ev[2], st);
      its++;
      // classical Gram-Schmidt, repeated once when the norm drops by > 1/sqrt(2)
      const int kk = j + 1;
      double *hd = W.hdev;  // [0..2kk) h, then norms
      if ((rc = bl.mdot(W.Vb, n, kk, W.w, n, hd, hd + 2 * 80, st))) return rc;
      if ((rc = bl.maxpy_norm(W.Vb, n, kk, hd, W.w, n, hd + 2 * 80 + 1, st))) return rc;
      DD_CUDA(cudaMemcpyAsync(bl.hpin, hd, sizeof(double) * (2 * 80 + 2), cudaMemcpyDeviceToHost, st));
      cudaEventRecord(W.ev[3], st);
      DD_CUDA(cudaStreamSynchronize(st));
      std::vector<cd> h(kk);
      for (int i = 0; i < kk; i++) h[i] = cd(bl.hpin[2 * i], bl.hpin[2 * i + 1]);
      double w0 = bl.hpin[160], w1 = bl.hpin[161];
      if (w1 < 0.5 * w0) {
        if ((rc = bl.mdot(W.Vb, n, kk, W.w, n, hd, nullptr, st))) return rc;
        if ((rc = bl.maxpy_norm(W.Vb, n, kk, hd, W.w, n, hd + 2 * 80 + 1, st))) return rc;
        DD_CUDA(cudaMemcpyAsync(bl.hpin, hd, sizeof(double) * (2 * 80 + 2), cudaMemcpyDeviceToHost, st));
        cudaEventRecord(W.ev[3], st);
        DD_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < kk; i++) h[i] += cd(bl.hpin[2 * i], bl.hpin[2 * i + 1]);
        w1 = bl.hpin[161];
      }
      ms_sap += ev_ms(W.ev[0], W.ev[1]);
      ms_dirac += ev_ms(W.ev[1], W.ev[2]);
      ms_orth += ev_ms(W.ev[2], W.ev[3]);
      double hn = std::sqrt(std::max(w1, 0.0));
      for (int i = 0; i < kk; i++) H[(size_t)i * m + j] = h[i];
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0 && j + 1 <= m)
        if ((rc = bl.scale(W.Vb + 2 * n * (j + 1), W.w, 1.0 / hn, n, st))) return rc;
      // Givens rotations
      for (int i = 0; i < j; i++) {
        cd a = H[(size_t)i * m + j], c2 = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c2;
        H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * c2;
      }
      cd a = H[(size_t)j * m + j];
      double bb = hn, rr = std::sqrt(std::norm(a) + bb * bb);
      if (std::abs(a) == 0) { cs[j] = 0; sn[j] = 1; }
      else { cs[j] = std::abs(a) / rr; sn[j] = (a / std::abs(a)) * bb / rr; }
      H[(size_t)j * m + j] = cs[j] * a + sn[j] * bb;
      H[(size_t)(j + 1) * m + j] = 0;
      gv[j + 1] = -std::conj(sn[j]) * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      est = std::abs(gv[j + 1]) / bnorm;
      if (std::abs(gv[j + 1]) <= target || hn == 0) break;
      if (cancel && *cancel) break;
    }
    // y = R^-1 g ; x += Z y
    for (int i = k - 1; i >= 0; i--) {
      cd s = gv[i];
      for (int l = i + 1; l < k; l++) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; i++) {
      bl.hpin[2 * i] = y[i].real();
      bl.hpin[2 * i + 1] = y[i].imag();
    }
    DD_CUDA(cudaMemcpyAsync(W.ydev, bl.hpin, sizeof(double) * 2 * k, cudaMemcpyHostToDevice, st));
    if ((rc = bl.update_x(g, W.x, W.zprec, W.Z, W.zbytes, k, W.ydev, st))) return rc;
  }
  DD_CUDA(cudaStreamSynchronize(st));
  info.status = status;
  info.iterations = its;
  info.true_rel_residual = rel;
  info.est_rel_residual = est;
  info.ms_sap = ms_sap;
  info.ms_dirac = ms_dirac;
  info.ms_orth = ms_orth;
  info.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return status == DD_ECANCELLED ? DD_ECANCELLED : DD_OK;
}

int check_solve_params(const dd_solve_params *p) {
  if (!p || !(p->tol > 0) || p->restart < 1 || p->restart > 64 || p->max_iter < 1 || p->sap.sweeps < 1 ||
      p->sap.mr_steps < 0 || p->inner_reduction < 0 || p->inner_reduction >= 1) {
    set_error("dd_solve: bad parameters (tol > 0, 1 <= restart <= 64, max_iter >= 1, sweeps >= 1)");
    return DD_EINVAL;
  }
  return DD_OK;
}

// Solve for nrhs canonical right-hand sides, one after the other.
int solve_canonical(const Op *op, const dd_solve_params &p, const double *b, double *x, int nrhs,
                    dd_solve_info *info, cudaStream_t st, SolveWork &W, const volatile int *cancel) {
  const Geom &g = op->lat->g;
  int rc = W.ensure(g, op->prec, p.restart);
  if (rc) return rc;
  const size_t fb = (size_t)g.V * 24 * sizeof(double);
  const cudaMemcpyKind h2d = p.where == DD_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind d2h = p.where == DD_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int all_ok = 1;
  for (int r = 0; r < nrhs; r++) {
    dd_solve_info inf{};
    DD_CUDA(cudaMemcpyAsync(W.canon, b + (size_t)r * g.V * 24, fb, h2d, st));
    if ((rc = launch_pack(g, DD_F64, W.canon, W.b, 1, 1.0, st))) return rc;
    if (p.use_x0) {
      DD_CUDA(cudaMemcpyAsync(W.canon, x + (size_t)r * g.V * 24, fb, h2d, st));
      if ((rc = launch_pack(g, DD_F64, W.canon, W.x, 1, 1.0, st))) return rc;
    } else {
      DD_CUDA(cudaMemsetAsync(W.x, 0, fb, st));
    }
    rc = fgmres_one(op, p, W, inf, st, cancel);
    if (rc && rc != DD_ECANCELLED) return rc;
    if ((rc = launch_unpack(g, DD_F64, W.x, W.canon, 1, 1.0, st))) return rc;
    DD_CUDA(cudaMemcpyAsync(x + (size_t)r * g.V * 24, W.canon, fb, d2h, st));
    DD_CUDA(cudaStreamSynchronize(st));
    if (info) info[r] = inf;
    if (inf.status == DD_ECANCELLED) return DD_ECANCELLED;
    if (inf.status != DD_OK) all_ok = 0;
  }
  if (!all_ok) {
    set_error("dd_solve: max_iter reached before the target residual");
    return DD_ENOTCONV;
  }
  return DD_OK;
}

}  // namespace dd

using namespace dd;

extern "C" int dd_solve(dd_op_t opp, const dd_solve_params *p, const double *b, double *x, int nrhs,
                        dd_solve_info *info, void *stream) {
  Op *op = (Op *)opp;
  if (!op || op->magic != 0x4f505231 || !b || !x || nrhs < 1) {
    set_error("dd_solve: bad argument");
    return DD_EINVAL;
  }
  int rc = check_solve_params(p);
  if (rc) return rc;
  SolveWork W;
  return solve_canonical(op, *p, b, x, nrhs, info, (cudaStream_t)stream, W, nullptr);
}
