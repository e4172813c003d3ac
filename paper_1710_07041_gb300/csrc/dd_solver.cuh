// Outer FGMRES solver internals (see dd_solver.cu).
#pragma once
#include <atomic>
#include <chrono>
#include <complex>
#include <functional>
#include <utility>
#include <vector>

#include "dd_mg.cuh"

namespace dd {

// One right-hand side to solve.
struct RhsJob {
  // operator of this right-hand side (null: the solver's own); any operator
  // with the solver operator's smoother precision and block shape
  const Op *op = nullptr;
  const double *b = nullptr;  // canonical FP64 right-hand side [V][4][3][2]
  int b_on_device = 0;
  double *x = nullptr;        // canonical FP64 solution (initial guess if use_x0)
  int x_on_device = 0;
  int use_x0 = 0;
  dd_solve_info *info = nullptr;      // result record (may be null)
  const std::atomic<int> *cancel = nullptr;
  std::function<void(int status)> done;  // called after x and info are written
};

// Device buffers and FGMRES state of one batch slot.
struct Slot {
  const Op *op = nullptr;   // operator of the right-hand side in the slot
  size_t f64 = 0, fz = 0, fp = 0;   // its field sizes (FP64, preconditioned vectors, smoother)
  long long vol = 0;        // lattice volume the slot's buffers were allocated for (0: none)
  double sigma = 1;         // smoother-input scale sqrt(24 V)
  bool busy = false, need_restart = true;
  bool x_zero = false;   // x is exactly zero (first cycle without an initial guess): r = b, no Dslash
  RhsJob job;
  int j = 0, its = 0, cycles = 0;
  double bnorm = -1, beta = 0, rel = 1, est = 1, target = 0;
  std::vector<std::complex<double>> H, g, sn, y;
  std::vector<double> cs;
  double ms_sap = 0, ms_dirac = 0, ms_orth = 0;
  std::chrono::steady_clock::time_point t0;
  // device memory
  double *Vb = nullptr;  // (m+1) basis fields: FP64, or double-float (float4 per complex)
  // double-float basis: vector i is stored unnormalised, v_i = scl[i] * Vb_i
  // (the Gram-Schmidt update writes it in place; no normalisation pass)
  std::vector<double> scl;
  double *sdev = nullptr;   // device scl[i]^2: the update coefficient of Vb_i is scl[i]^2 <Vb_i, w>
  char *Z = nullptr;     // m preconditioned fields (zprec)
  double *x = nullptr, *b = nullptr, *w = nullptr, *canon = nullptr;
  void *tin = nullptr, *tout = nullptr, *zt = nullptr;
  void *se = nullptr, *sr = nullptr;   // smoother work fields (corrections, block residuals)
  MgWork *mgw = nullptr;   // coarse-solve workspace when preconditioning with multigrid
};

// FGMRES(m) right-preconditioned by SAP over a batch of right-hand sides:
// the slots' Schwarz sweeps run as single launches (also across operators
// on different lattices, as long as they share the smoother precision and
// block shape), the Dslash products as one launch per operator,
// orthogonalisation and Givens rotations per slot. Slots retire when their
// right-hand side converges and are refilled from the job source at the next
// Arnoldi step (continuous batching); a slot's buffers are resized when it
// takes a right-hand side on a lattice of another size.
class BatchSolver {
 public:
  BatchSolver(const Op *op, const dd_solve_params &p, int slots, cudaStream_t st);
  ~BatchSolver();
  int init();
  // Device bytes one slot needs for this lattice, precision and restart.
  static size_t bytes_per_slot(const Geom &g, int prec, int m);
  // Solve jobs until next() returns false and every slot has retired.
  int run(const std::function<bool(RhsJob &)> &next);
  int nslots() const { return (int)slots_.size(); }
  const Op *op() const { return op_; }
  const dd_solve_params &params() const { return p_; }
  void set_params(const dd_solve_params &p) { p_ = p; }
  // false: the destructor frees the workspace instead of caching it for reuse
  void set_cache_workspace(bool on) { cache_ = on; }

 private:
  int start(Slot &s);
  int size_slot(Slot &s, const Op *op);   // buffers of slot s for right-hand sides of op
  int free_slot(Slot &s);
  int restart_phase(std::vector<Slot *> &R);
  int arnoldi_step(std::vector<Slot *> &A);
  int end_cycle(Slot &s);
  int retire(Slot &s, int status);
  int sync_h();
  // the slot's buffers with their sizes for lattice volume V (allocation and
  // release walk the same list)
  std::vector<std::pair<void **, size_t>> slot_buffers(Slot &s, long long V) const;
  int mdot(Slot *s, int kk, double *h, double *wn2, bool from32 = false);
  int maxpy(Slot *s, int kk, const double *h, double *wn2, bool from32 = false);

  const Op *op_;
  dd_solve_params p_;
  cudaStream_t st_;
  std::vector<Slot> slots_;
  int zprec_;
  bool df_;  // Krylov basis and w in double-float

  Blas blas_;
  double *hdev_ = nullptr;   // [slots][HSTRIDE]
  double *hpin_ = nullptr;   // pinned mirror [slots][HSTRIDE]
  double *ydev_ = nullptr;   // [slots][2*64]
  double *ypin_ = nullptr;
  cudaEvent_t ev_[4] = {};
  cudaStream_t caller_ = nullptr;  // the caller's stream
  bool own_stream_ = false;        // st_ created here (the caller passed the legacy stream)
  int failed_ = 0;
  bool cache_ = true;   // release the workspace into the cache (dd_pool.cu)
  int m_alloc_ = 0;     // restart length the slot buffers were sized for
};

constexpr int HSTRIDE = 2 * 65 + 6;  // h column (complex) + norms

// Classical Gram-Schmidt is repeated only when the new vector's squared norm
// falls below REORTH2 times its value before the projection (norm ratio
// 1e-3). One pass then loses orthogonality by at most ~eps / 1e-3: about 1e-11
// with the double-float or FP64 arithmetic used here, far below the 1e-5 to
// 1e-7 reduction a cycle asks for, while the classic 1/sqrt(2) test would
// repeat nearly every step of a well-preconditioned solve.
constexpr double REORTH2 = 1e-6;

int check_solve_params(const dd_solve_params *p);

}  // namespace dd
