// Outer solver: FGMRES(m) right-preconditioned by the Schwarz method
// (Saad 1993). The paper calls DD-alpha-AMG for the Dirac equation (Sec. 1)
// with SAP as its fine-grid smoother (Sec. 3.1); this library runs the
// SAP-preconditioned fine-grid Krylov solve, with mixed precision in the
// spirit of Sec. 3.1's half-precision storage: the smoother works in the
// operator's storage precision, while the Arnoldi orthogonalisation, the
// least-squares update and the true residual are FP64-class: IEEE FP64 for
// an FP64 operator; for a mixed-precision one the Krylov basis and the true
// residual's Dslash use double-float arithmetic (FP32 pairs, ~48-bit
// significands, on GB300's FP32 pipes), the least-squares update, x and the
// residual's inputs and outputs stay FP64. Preconditioned vectors z_j are
// kept in FP32 (FP64 for an FP64 operator) and the Arnoldi product D z_j uses
// the operator in that same precision, so D Z = V H holds to that precision;
// each cycle ends with the true residual, so restarts act as iterative
// refinement.
//
// Batching: right-hand sides that share an operator occupy the slots of one
// BatchSolver. Per Arnoldi step all slots' Schwarz sweeps are one launch per
// colour phase and all Dslash products one launch; each slot's reductions,
// Givens rotations and convergence decisions are its own, so a right-hand
// side gets bit-identical results alone or in any mix.
#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "dd_solver.cuh"
#include "dd_pool.cuh"

namespace dd {

using cd = std::complex<double>;
namespace {
constexpr int W0 = 130, W1 = 131, RN = 132, BN = 133;

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float t = 0;
  cudaEventElapsedTime(&t, a, b);
  return t;
}
}  // namespace

int check_solve_params(const dd_solve_params *p) {
  if (!p || !(p->tol > 0) || p->restart < 1 || p->restart > 64 || p->max_iter < 1 || p->sap.sweeps < 1 ||
      p->sap.mr_steps < 0 || !(p->inner_reduction >= 0) || p->inner_reduction >= 1 || p->outer_f64 < 0 ||
      p->outer_f64 > 1 || (p->outer_f64 && p->mg)) {
    set_error("dd_solve: bad parameters (tol > 0, 1 <= restart <= 64, max_iter >= 1, sweeps >= 1, "
              "0 <= inner_reduction < 1, outer_f64 0 or 1 and not with mg)");
    return DD_EINVAL;
  }
  return DD_OK;
}

size_t BatchSolver::bytes_per_slot(const Geom &g, int prec, int m) {
  size_t f64 = (size_t)g.V * 24 * 8;
  int zprec = prec == DD_F64 ? DD_F64 : DD_F32;
  size_t fz = (size_t)g.V * spinor_site_bytes(zprec), fp = (size_t)g.V * spinor_site_bytes(prec);
  return (size_t)(m + 1) * f64 + (size_t)m * fz + 4 * f64 + 4 * fp + fz;
}

BatchSolver::BatchSolver(const Op *op, const dd_solve_params &p, int slots, cudaStream_t st)
    : op_(op), p_(p), st_(st), slots_(slots), caller_(st) {
  zprec_ = op->prec == DD_F64 ? DD_F64 : DD_F32;
  // mixed precision keeps the Krylov basis in double-float (FP32 hi/lo pairs):
  // FP64-class accuracy at FP32 ALU rate; an FP64 operator keeps native FP64
  df_ = zprec_ == DD_F32 && !p.outer_f64;
}

// The device buffers of one slot with their sizes (allocation and release
// walk the same list).
std::vector<std::pair<void **, size_t>> BatchSolver::slot_buffers(Slot &s, long long V) const {
  const size_t m = (size_t)m_alloc_;
  const size_t f64 = (size_t)V * 24 * 8, fz = (size_t)V * spinor_site_bytes(zprec_),
               fp = (size_t)V * spinor_site_bytes(op_->prec);
  return {{(void **)&s.Vb, (m + 1) * f64}, {(void **)&s.Z, m * fz},   {(void **)&s.x, f64},
          {(void **)&s.b, f64},           {(void **)&s.w, f64},       {(void **)&s.canon, f64},
          {&s.tin, fp},                   {&s.tout, fp},              {&s.zt, fz},
          {&s.se, fp},                    {&s.sr, fp},
          {(void **)&s.sdev, sizeof(double) * (m + 1)}};
}

// Release slot s's field buffers (to the workspace cache, or to the device).
int BatchSolver::free_slot(Slot &s) {
  if (!s.vol) return DD_OK;
  if (cache_) {
    DD_CUDA(cudaStreamSynchronize(st_));   // queued work may still use them
    for (auto &pb : slot_buffers(s, s.vol)) pool_dev_free(*pb.first, pb.second);
  } else {
    for (auto &pb : slot_buffers(s, s.vol))
      if (*pb.first) cudaFree(*pb.first);
  }
  for (auto &pb : slot_buffers(s, s.vol)) *pb.first = nullptr;
  s.vol = 0;
  return DD_OK;
}

// Give slot s buffers for right-hand sides of op. Buffers only grow: a
// lattice no larger than the slot's allocation reuses it (releasing device
// memory synchronises the whole device, which would stall the other
// workers' streams at every change of lattice).
int BatchSolver::size_slot(Slot &s, const Op *op) {
  bool same_shape = op->prec == op_->prec;
  for (int mu = 0; mu < 4; mu++) same_shape = same_shape && op->lat->g.bd[mu] == op_->lat->g.bd[mu];
  if (!same_shape || (p_.mg && op != op_)) {
    set_error("solver: a batch mixes operators of different smoother precision or block shape");
    return DD_EINVAL;
  }
  const Geom &g = op->lat->g;
  s.op = op;
  s.f64 = (size_t)g.V * 24 * 8;
  s.fz = (size_t)g.V * spinor_site_bytes(zprec_);
  s.fp = (size_t)g.V * spinor_site_bytes(op->prec);
  s.sigma = std::sqrt(24.0 * (double)g.V);  // unit-norm vector -> unit RMS entries
  if (s.vol >= g.V) return DD_OK;
  int rc = free_slot(s);
  if (rc) return rc;
  s.vol = g.V;
  for (auto &pb : slot_buffers(s, s.vol))
    if (!(*pb.first = pool_dev_alloc(pb.second))) {
      set_error("solver: out of device memory for an FGMRES(%d) slot (%zu bytes)", m_alloc_,
                bytes_per_slot(g, op->prec, m_alloc_));
      return DD_ENOMEM;
    }
  return DD_OK;
}

BatchSolver::~BatchSolver() {
  if (cache_) {
    // the workspace goes back to the cache, so no queued work may still use it
    cudaStreamSynchronize(st_);
    const size_t n = slots_.size();
    for (auto &s : slots_)
      if (s.vol)
        for (auto &pb : slot_buffers(s, s.vol)) pool_dev_free(*pb.first, pb.second);
    pool_dev_free(hdev_, sizeof(double) * HSTRIDE * n);
    pool_dev_free(ydev_, sizeof(double) * 2 * 64 * n);
    pool_host_free(hpin_, sizeof(double) * HSTRIDE * n);
    pool_host_free(ypin_, sizeof(double) * 2 * 64 * n);
    blas_.release_to_pool();
  } else {
    for (auto &s : slots_)
      if (s.vol)
        for (auto &pb : slot_buffers(s, s.vol))
          if (*pb.first) cudaFree(*pb.first);
    if (hdev_) cudaFree(hdev_);
    if (ydev_) cudaFree(ydev_);
    if (hpin_) cudaFreeHost(hpin_);
    if (ypin_) cudaFreeHost(ypin_);
  }
  for (auto &s : slots_) delete s.mgw;
  for (auto &e : ev_)
    if (e) cudaEventDestroy(e);
  if (own_stream_) cudaStreamDestroy(st_);
}

int BatchSolver::init() {
  const int m = p_.restart, n = (int)slots_.size();
  m_alloc_ = m;
  if (n < 1 || n > MAX_RHS) {
    set_error("solver: 1..%d slots", MAX_RHS);
    return DD_EINVAL;
  }
  for (auto &s : slots_) {
    // buffers for the solver's own operator up front (a slot is resized when
    // it takes a right-hand side on a lattice of another volume)
    int rc = size_slot(s, op_);
    s.scl.assign(m + 1, 1.0);
    if (rc == DD_ENOMEM)
      set_error("solver: out of device memory for %d FGMRES(%d) slots (%zu bytes each)", n, m,
                bytes_per_slot(op_->lat->g, op_->prec, m));
    if (rc) return rc;
    if (p_.mg) {
      s.mgw = new (std::nothrow) MgWork;
      int rc = s.mgw ? s.mgw->init((const Mg *)p_.mg) : DD_ENOMEM;
      if (rc) return rc;
    }
    s.H.assign((size_t)(m + 1) * m, 0);
    s.g.assign(m + 1, 0);
    s.sn.assign(m, 0);
    s.y.assign(m, 0);
    s.cs.assign(m, 0);
  }
  hdev_ = (double *)pool_dev_alloc(sizeof(double) * HSTRIDE * n);
  ydev_ = (double *)pool_dev_alloc(sizeof(double) * 2 * 64 * n);
  hpin_ = (double *)pool_host_alloc(sizeof(double) * HSTRIDE * n);
  ypin_ = (double *)pool_host_alloc(sizeof(double) * 2 * 64 * n);
  if (!hdev_ || !ydev_ || !hpin_ || !ypin_) {
    set_error("solver: out of memory for the Hessenberg buffers");
    return DD_ENOMEM;
  }
  for (auto &e : ev_) DD_CUDA(cudaEventCreate(&e));
  // work on a stream of our own when given the legacy default stream, so the
  // smoother's launches can be captured into CUDA graphs
  if (caller_ == nullptr) {
    DD_CUDA(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return blas_.init(sms);
}

int BatchSolver::sync_h() {
  DD_CUDA(cudaMemcpyAsync(hpin_, hdev_, sizeof(double) * HSTRIDE * slots_.size(), cudaMemcpyDeviceToHost, st_));
  return cuda_fail(cudaStreamSynchronize(st_), "solver sync");
}

// Load a job into a slot: b and x0 into the FP64 field layout.
int BatchSolver::start(Slot &s) {
  int rc = size_slot(s, s.job.op ? s.job.op : op_);
  if (rc) return rc;
  const Geom &g = s.op->lat->g;
  const size_t f64_ = s.f64;
  s.busy = true;
  s.need_restart = true;
  s.j = s.its = s.cycles = 0;
  s.bnorm = -1;
  s.rel = s.est = 1;
  s.ms_sap = s.ms_dirac = s.ms_orth = 0;
  s.t0 = std::chrono::steady_clock::now();
  DD_CUDA(cudaMemcpyAsync(s.canon, s.job.b, f64_, s.job.b_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          st_));
  if ((rc = launch_pack(g, DD_F64, s.canon, s.b, 1, 1.0, st_))) return rc;
  s.x_zero = !s.job.use_x0;
  if (s.job.use_x0) {
    DD_CUDA(cudaMemcpyAsync(s.canon, s.job.x, f64_,
                            s.job.x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st_));
    if ((rc = launch_pack(g, DD_F64, s.canon, s.x, 1, 1.0, st_))) return rc;
  } else {
    DD_CUDA(cudaMemsetAsync(s.x, 0, f64_, st_));
  }
  return DD_OK;
}

int BatchSolver::retire(Slot &s, int status) {
  const Geom &g = s.op->lat->g;
  const size_t f64_ = s.f64;
  int rc;
  if ((rc = launch_unpack(g, DD_F64, s.x, s.canon, 1, 1.0, st_))) return rc;
  DD_CUDA(cudaMemcpyAsync(s.job.x, s.canon, f64_, s.job.x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          st_));
  DD_CUDA(cudaStreamSynchronize(st_));
  if (s.job.info) {
    dd_solve_info &inf = *s.job.info;
    inf.status = status;
    inf.iterations = s.its;
    inf.cycles = s.cycles;
    inf.true_rel_residual = s.rel;
    inf.est_rel_residual = s.est;
    inf.ms_sap = s.ms_sap;
    inf.ms_dirac = s.ms_dirac;
    inf.ms_orth = s.ms_orth;
    inf.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - s.t0).count();
  }
  if (status != DD_OK) failed_ = 1;
  s.busy = false;
  if (s.job.done) s.job.done(status);
  return DD_OK;
}

// True residual r = b - D x (FP64) for the slots in R; retire or begin a cycle.
// The slots of S grouped by operator, groups in order of first appearance.
static std::vector<std::vector<Slot *>> by_operator(const std::vector<Slot *> &S) {
  std::vector<std::vector<Slot *>> groups;
  for (Slot *s : S) {
    size_t k = 0;
    while (k < groups.size() && groups[k][0]->op != s->op) k++;
    if (k == groups.size()) groups.emplace_back();
    groups[k].push_back(s);
  }
  return groups;
}

int BatchSolver::restart_phase(std::vector<Slot *> &R) {
  NvtxRange range("dd:true_residual");
  int rc;
  // D x for the slots whose x is not known to be zero (w = 0 for the others,
  // so that w = b - w below gives r = b), one launch per operator.
  // In a mixed-precision solve the Dslash runs in double-float arithmetic on
  // the operator's pre-split fields: x is split into the slot's staging
  // buffer (free at this point; FP64 field size); the result stays FP64.
  cudaEventRecord(ev_[0], st_);
  for (auto &grp : by_operator(R)) {
    const Op *op = grp[0]->op;
    const Geom &g = op->lat->g;
    const size_t n = (size_t)g.V * 12;
    RhsPtrs rp;
    rp.n = 0;
    for (Slot *s : grp) {
      if (s->x_zero) {
        DD_CUDA(cudaMemsetAsync(s->w, 0, s->f64, st_));
        s->x_zero = false;
        continue;
      }
      if (df_ && (rc = launch_split_pairs(s->x, s->canon, n, st_))) return rc;
      rp.in[rp.n] = df_ ? (const void *)s->canon : (const void *)s->x;
      rp.out[rp.n++] = s->w;
    }
    if (rp.n && (rc = df_ ? launch_dirac_df(g, op->fdf, rp, st_) : launch_dirac(g, op->f64, rp, st_))) return rc;
  }
  for (Slot *s : R) {
    const size_t n = (size_t)s->op->lat->g.V * 12;
    double *hd = hdev_ + HSTRIDE * (s - slots_.data());
    if ((rc = blas_.xmy(s->b, s->w, n, st_))) return rc;
    if ((rc = blas_.norm2(s->w, n, hd + RN, st_))) return rc;
    if (s->bnorm < 0 && (rc = blas_.norm2(s->b, n, hd + BN, st_))) return rc;
  }
  cudaEventRecord(ev_[1], st_);
  if ((rc = sync_h())) return rc;
  float ms = ev_ms(ev_[0], ev_[1]);
  for (Slot *s : R) {
    const double *hp = hpin_ + HSTRIDE * (s - slots_.data());
    s->ms_dirac += ms;
    if (s->bnorm < 0) s->bnorm = std::sqrt(hp[BN]);
    s->beta = std::sqrt(hp[RN]);
    s->rel = s->bnorm > 0 ? s->beta / s->bnorm : 0.0;
    if (s->bnorm == 0) {
      DD_CUDA(cudaMemsetAsync(s->x, 0, s->f64, st_));
      s->est = 0;
      if ((rc = retire(*s, DD_OK))) return rc;
      continue;
    }
    if (!std::isfinite(s->rel)) {
      if ((rc = retire(*s, DD_ENOTCONV))) return rc;
      continue;
    }
    if (s->rel <= p_.tol) {
      s->est = s->rel;
      if ((rc = retire(*s, DD_OK))) return rc;
      continue;
    }
    if (s->job.cancel && *s->job.cancel) {
      if ((rc = retire(*s, DD_ECANCELLED))) return rc;
      continue;
    }
    if (s->its >= p_.max_iter) {
      if ((rc = retire(*s, DD_ENOTCONV))) return rc;
      continue;
    }
    s->cycles++;
    s->need_restart = false;
    s->j = 0;
    std::fill(s->g.begin(), s->g.end(), cd(0));
    s->g[0] = s->beta;
    s->target = std::max(p_.tol * s->bnorm, p_.inner_reduction * s->beta);
    const size_t n = (size_t)s->op->lat->g.V * 12;
    if (df_) {
      rc = blas_.f64_to_df((float *)s->Vb, s->w, 1.0 / s->beta, n, st_);
      s->scl[0] = 1.0;
      if (rc == DD_OK) rc = blas_.set_double(s->sdev, 1.0, st_);
    } else {
      rc = blas_.scale(s->Vb, s->w, 1.0 / s->beta, n, st_);
    }
    if (rc) return rc;
  }
  return DD_OK;
}

int BatchSolver::end_cycle(Slot &s) {
  const Geom &g = s.op->lat->g;
  const int m = p_.restart, k = s.j + 1;
  for (int i = k - 1; i >= 0; i--) {
    cd t = s.g[i];
    for (int l = i + 1; l < k; l++) t -= s.H[(size_t)i * m + l] * s.y[l];
    s.y[i] = t / s.H[(size_t)i * m + i];
  }
  const int idx = (int)(&s - slots_.data());
  double *yp = ypin_ + 2 * 64 * idx;
  double *yd = ydev_ + 2 * 64 * idx;
  for (int i = 0; i < k; i++) {
    yp[2 * i] = s.y[i].real();
    yp[2 * i + 1] = s.y[i].imag();
  }
  DD_CUDA(cudaMemcpyAsync(yd, yp, sizeof(double) * 2 * k, cudaMemcpyHostToDevice, st_));
  int rc = blas_.update_x(g, s.x, zprec_, s.Z, s.fz, k, yd, st_);
  s.need_restart = true;
  return rc;
}

// Double-float solves: the first Gram-Schmidt pass reads w = D z_j from the
// FP32 field s->zt (from32) and maxpy writes the result straight into the
// basis slot j+1 (kk = j+1); the re-orthogonalisation pass works on that
// slot. The dots h_i = <Vb_i, w> are taken against the stored
// (unnormalised) vectors; the Hessenberg entry is scl[i] h_i and the update
// w -= <v_i, w> v_i applies scl[i]^2 h_i to Vb_i (sdev). FP64 solves use s->w.
int BatchSolver::mdot(Slot *s, int kk, double *h, double *wn2, bool from32) {
  const Geom &g = s->op->lat->g;
  const size_t n = (size_t)g.V * 12;
  const int lvb = g.lbd[0] + g.lbd[1] + g.lbd[2] + g.lbd[3];
  if (df_)
    return blas_.df_mdot((const float *)s->Vb, n, kk, (const float *)(s->Vb + 2 * n * kk), n, h, wn2, st_,
                         from32 ? (const float *)s->zt : nullptr, lvb);
  return blas_.mdot(s->Vb, n, kk, s->w, n, h, wn2, st_);
}

int BatchSolver::maxpy(Slot *s, int kk, const double *h, double *wn2, bool from32) {
  const Geom &g = s->op->lat->g;
  const size_t n = (size_t)g.V * 12;
  const int lvb = g.lbd[0] + g.lbd[1] + g.lbd[2] + g.lbd[3];
  if (df_)
    return blas_.df_maxpy_norm((const float *)s->Vb, n, kk, h, (float *)(s->Vb + 2 * n * kk), n, wn2, st_,
                               from32 ? (const float *)s->zt : nullptr, lvb, s->sdev);
  return blas_.maxpy_norm(s->Vb, n, kk, h, s->w, n, wn2, st_);
}

// One preconditioned Arnoldi step for every slot in A.
int BatchSolver::arnoldi_step(std::vector<Slot *> &A) {
  NvtxRange range("dd:arnoldi_step");
  const int m = p_.restart;
  int rc;
  // the slots by operator (lattice): each group is one lattice of the
  // smoother's launch and one Dslash launch
  const std::vector<std::vector<Slot *>> groups = by_operator(A);
  // z_j = SAP(sigma v_j) in zprec. z_j is kept scaled by sigma (the smoother
  // input's scale): then w = D z_j, the Hessenberg column and y carry the same
  // factor and x += Z y is unchanged, with no rescaling pass.
  cudaEventRecord(ev_[0], st_);
  if (p_.mg) {
    // two-level preconditioner per slot (FP32): z_j = M (sigma v_j) / sigma
    for (Slot *s : A) {
      const Geom &g = s->op->lat->g;
      const size_t n = (size_t)g.V * 12;
      char *zj = s->Z + (size_t)s->j * s->fz;
      if ((rc = blas_.df_to_field(g, (const float *)(s->Vb + 2 * n * s->j), DD_F32, s->zt, s->sigma * s->scl[s->j],
                                  st_)))
        return rc;
      if ((rc = mg_apply((const Mg *)p_.mg, *s->mgw, (const float *)s->zt, (float *)zj, st_, 1.f))) return rc;
    }
  } else {
    const bool direct = op_->prec == zprec_ && A.size() == 1;
    RhsPtrs sp_ptrs;
    AuxPtrs ax;
    SapLattice lats[MAX_SAP_GROUPS];
    int nlat = 0;
    sp_ptrs.n = 0;
    dd_sap_params sp = p_.sap;
    sp.x_is_zero = 1;
    for (size_t k = 0; k < groups.size(); k++) {
      for (Slot *s : groups[k]) {
        const Geom &g = s->op->lat->g;
        const size_t n = (size_t)g.V * 12;
        if (df_)
          rc = blas_.df_to_field(g, (const float *)(s->Vb + 2 * n * s->j), s->op->prec, s->tin,
                                 s->sigma * s->scl[s->j], st_);
        else rc = launch_convert_field(g, DD_F64, s->Vb + 2 * n * s->j, s->op->prec, s->tin, 1, s->sigma, st_);
        if (rc) return rc;
        // a single slot's smoother writes z_j straight into Z when it works in
        // Z's precision (with several slots the fixed output buffers keep the
        // smoother's graph cache to one entry per slot set; the copy below is
        // exact, so results are the same either way)
        const int i = sp_ptrs.n++;
        sp_ptrs.in[i] = s->tin;
        sp_ptrs.out[i] = direct ? (void *)(s->Z + (size_t)s->j * s->fz) : s->tout;
        ax.e[i] = s->se;
        ax.r[i] = s->sr;
      }
      lats[nlat++] = SapLattice{groups[k][0]->op->lat->g, groups[k][0]->op->fp, (int)groups[k].size()};
      // one launch per MAX_SAP_GROUPS lattices
      if (nlat == MAX_SAP_GROUPS || k + 1 == groups.size()) {
        if ((rc = launch_sap_lattices(lats, nlat, sp, sp_ptrs, st_, &ax))) return rc;
        nlat = 0;
        sp_ptrs.n = 0;
      }
    }
    for (Slot *s : A) {
      char *zj = s->Z + (size_t)s->j * s->fz;
      if (!direct && (rc = launch_convert_field(s->op->lat->g, s->op->prec, s->tout, zprec_, zj, 1, 1.0, st_)))
        return rc;
    }
  }
  cudaEventRecord(ev_[1], st_);
  // w = D z_j in zprec, one launch per operator (a double-float solve keeps it
  // in the FP32 field zt; the first Gram-Schmidt pass reads it there and
  // writes the DF w)
  for (auto &grp : groups) {
    const Op *op = grp[0]->op;
    RhsPtrs d_ptrs;
    d_ptrs.n = 0;
    for (Slot *s : grp) {
      d_ptrs.in[d_ptrs.n] = s->Z + (size_t)s->j * s->fz;
      d_ptrs.out[d_ptrs.n++] = (zprec_ == DD_F64 && !p_.mg) ? (void *)s->w : s->zt;
    }
    if ((rc = launch_dirac(op->lat->g, zprec_ == DD_F64 ? op->f64 : op->f32, d_ptrs, st_))) return rc;
  }
  // an IEEE FP64 basis with FP32 preconditioned vectors (outer_f64): w = D z_j as FP64
  if (!df_ && zprec_ != DD_F64)
    for (Slot *s : A)
      if ((rc = launch_convert_field(s->op->lat->g, zprec_, s->zt, DD_F64, s->w, 1, 1.0, st_))) return rc;
  cudaEventRecord(ev_[2], st_);
  // classical Gram-Schmidt, repeated once for slots whose norm drops below 1e-3 of its value (REORTH2)
  for (Slot *s : A) {
    double *hd = hdev_ + HSTRIDE * (s - slots_.data());
    const int kk = s->j + 1;
    if ((rc = mdot(s, kk, hd, hd + W0, df_))) return rc;
    if ((rc = maxpy(s, kk, hd, hd + W1, df_))) return rc;
  }
  if ((rc = sync_h())) return rc;
  std::vector<std::vector<cd>> hcol(A.size());
  std::vector<Slot *> again;
  for (size_t i = 0; i < A.size(); i++) {
    Slot *s = A[i];
    const double *hp = hpin_ + HSTRIDE * (s - slots_.data());
    hcol[i].resize(s->j + 1);
    for (int q = 0; q <= s->j; q++) hcol[i][q] = cd(hp[2 * q], hp[2 * q + 1]) * (df_ ? s->scl[q] : 1.0);
    if (hp[W1] < REORTH2 * hp[W0]) again.push_back(s);
  }
  if (!again.empty()) {
    for (Slot *s : again) {
      double *hd = hdev_ + HSTRIDE * (s - slots_.data());
      const int kk = s->j + 1;
      if ((rc = mdot(s, kk, hd, nullptr))) return rc;
      if ((rc = maxpy(s, kk, hd, hd + W1))) return rc;
    }
    if ((rc = sync_h())) return rc;
    for (size_t i = 0; i < A.size(); i++) {
      Slot *s = A[i];
      bool re = false;
      for (Slot *t : again) re |= t == s;
      if (!re) continue;
      const double *hp = hpin_ + HSTRIDE * (s - slots_.data());
      for (int q = 0; q <= s->j; q++) hcol[i][q] += cd(hp[2 * q], hp[2 * q + 1]) * (df_ ? s->scl[q] : 1.0);
    }
  }
  cudaEventRecord(ev_[3], st_);
  cudaEventSynchronize(ev_[3]);
  const float t_sap = ev_ms(ev_[0], ev_[1]), t_d = ev_ms(ev_[1], ev_[2]), t_o = ev_ms(ev_[2], ev_[3]);
  for (size_t i = 0; i < A.size(); i++) {
    Slot &s = *A[i];
    const double *hp = hpin_ + HSTRIDE * (&s - slots_.data());
    s.ms_sap += t_sap;
    s.ms_dirac += t_d;
    s.ms_orth += t_o;
    s.its++;
    const int j = s.j;
    const double hn = std::sqrt(std::max(hp[W1], 0.0));
    const size_t n = (size_t)s.op->lat->g.V * 12;
    for (int q = 0; q <= j; q++) s.H[(size_t)q * m + j] = hcol[i][q];
    if (hn > 0) {
      if (df_) {   // v_{j+1} = Vb_{j+1} / hn, kept as a scale
        s.scl[j + 1] = 1.0 / hn;
        rc = blas_.set_double(s.sdev + j + 1, 1.0 / (hn * hn), st_);
      } else {
        rc = blas_.scale(s.Vb + 2 * n * (j + 1), s.w, 1.0 / hn, n, st_);
      }
      if (rc) return rc;
    }
    for (int q = 0; q < j; q++) {
      cd a = s.H[(size_t)q * m + j], c2 = s.H[(size_t)(q + 1) * m + j];
      s.H[(size_t)q * m + j] = s.cs[q] * a + s.sn[q] * c2;
      s.H[(size_t)(q + 1) * m + j] = -std::conj(s.sn[q]) * a + s.cs[q] * c2;
    }
    cd a = s.H[(size_t)j * m + j];
    double rr = std::sqrt(std::norm(a) + hn * hn);
    if (std::abs(a) == 0) {
      s.cs[j] = 0;
      s.sn[j] = 1;
    } else {
      s.cs[j] = std::abs(a) / rr;
      s.sn[j] = (a / std::abs(a)) * hn / rr;
    }
    s.H[(size_t)j * m + j] = s.cs[j] * a + s.sn[j] * hn;
    s.g[j + 1] = -std::conj(s.sn[j]) * s.g[j];
    s.g[j] = s.cs[j] * s.g[j];
    s.est = std::abs(s.g[j + 1]) / s.bnorm;
    bool cancel = s.job.cancel && *s.job.cancel;
    if (std::abs(s.g[j + 1]) <= s.target || j + 1 == m || s.its >= p_.max_iter || hn == 0 || cancel) {
      if ((rc = end_cycle(s))) return rc;
    } else {
      s.j++;
    }
  }
  return DD_OK;
}

int BatchSolver::run(const std::function<bool(RhsJob &)> &next) {
  failed_ = 0;
  bool more = true;
  int rc;
  if (own_stream_) {   // order our stream after the caller's prior work
    DD_CUDA(cudaEventRecord(ev_[0], caller_));
    DD_CUDA(cudaStreamWaitEvent(st_, ev_[0], 0));
  }
  for (;;) {
    for (auto &s : slots_) {
      if (s.busy || !more) continue;
      RhsJob job;
      if (!next(job)) {
        more = false;
        break;
      }
      s.job = job;
      if ((rc = start(s))) return rc;
    }
    std::vector<Slot *> R, A;
    for (auto &s : slots_)
      if (s.busy && s.need_restart) R.push_back(&s);
    if (!R.empty() && (rc = restart_phase(R))) return rc;
    for (auto &s : slots_)
      if (s.busy && !s.need_restart) A.push_back(&s);
    if (A.empty()) {
      bool any = false;
      for (auto &s : slots_) any |= s.busy;
      if (!any && !more) break;
      continue;
    }
    if ((rc = arnoldi_step(A))) return rc;
  }
  if (own_stream_) {   // and the caller's later work after ours
    DD_CUDA(cudaEventRecord(ev_[0], st_));
    DD_CUDA(cudaStreamWaitEvent(caller_, ev_[0], 0));
  }
  return failed_ ? DD_ENOTCONV : DD_OK;
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
  if (p->mg && (((Mg *)p->mg)->magic != MAGIC_MG || ((Mg *)p->mg)->op != op || op->prec == DD_F64)) {
    set_error("dd_solve: the multigrid object must belong to this operator (FP32/FP16/BF16 smoother)");
    return DD_EINVAL;
  }
  const Geom &g = op->lat->g;
  // as many slots as right-hand sides, bounded by free device memory
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  free_b += pool_cached_bytes();   // cached workspaces are reused or released
  size_t per = BatchSolver::bytes_per_slot(g, op->prec, p->restart);
  if (p->mg) per += MgWork::bytes(g, op->prec, ((Mg *)p->mg)->N, ((Mg *)p->mg)->p.coarse_max_iter);
  int slots = nrhs < MAX_RHS ? nrhs : MAX_RHS;
  while (slots > 1 && (size_t)slots * per > free_b / 10 * 9) slots--;
  BatchSolver bs(op, *p, slots, (cudaStream_t)stream);
  if ((rc = bs.init())) return rc;
  int next = 0;
  std::vector<dd_solve_info> tmp(nrhs);
  rc = bs.run([&](RhsJob &j) {
    if (next >= nrhs) return false;
    j.b = b + (size_t)next * g.V * 24;
    j.x = x + (size_t)next * g.V * 24;
    j.b_on_device = j.x_on_device = p->where == DD_DEVICE;
    j.use_x0 = p->use_x0;
    j.info = info ? info + next : &tmp[next];
    next++;
    return true;
  });
  if (rc == DD_ENOTCONV) set_error("dd_solve: max_iter reached before the target residual");
  return rc;
}
