/*
 * dd.h - C ABI of the GB300 Wilson-clover SAP-FGMRES library (sm_103a).
 *
 * What it computes. The paper (arXiv:1710.07041, "DD-alpha-AMG on QPACE 3")
 * ports the DD-alpha-AMG solver for "the discretized form of the Dirac
 * equation" (Sec. 1); its two hot code parts are "the MR inversion within a
 * domain" (Sec. 3.1, Table 1) and "the entire Schwarz method" (Sec. 3.1,
 * Table 2), the fine-grid smoother, with some data stored in half precision
 * (Sec. 3, Listing 1: round-to-nearest conversion). The paper does not print
 * the formulas; this library implements the standard ones:
 *
 *   (D psi)(n) = A(n) psi(n)
 *       - 1/2 sum_mu [(1 - g_mu) U_mu(n) psi(n+mu) + (1 + g_mu) U_mu(n-mu)^+ psi(n-mu)]
 *   A(n) = (4 + m0) + C(n),
 *   C(n) = -(c_sw/32) sum_{mu,nu} g_mu g_nu (x) (Q_mu,nu(n) - Q_nu,mu(n)),
 *
 * Q_mu,nu the four-leaf clover sum; chiral gamma basis g_k = [[0,-i s_k],[i s_k,0]],
 * g_t = [[0,1],[1,0]]; periodic space, antiperiodic time (optional). The
 * smoother is red-black multiplicative Schwarz over lattice blocks, each block
 * solved by even-odd (odd-site Schur complement) minimal-residual steps; the
 * outer solver is FGMRES(m) right-preconditioned by it, with its Arnoldi
 * orthogonalisation, least-squares update and true residual in FP64-class
 * arithmetic (IEEE FP64, or double-float FP32 pairs where dd_solve says so).
 *
 * Conventions.
 *   dims  = {T, Z, Y, X}; canonical site n = x + X*(y + Y*(z + Z*t)).
 *   block = {bt, bz, by, bx}: Schwarz block and storage tile; each extent a
 *           power of two >= 2, dividing the lattice, with an even number of
 *           blocks in every direction (red-black colouring).
 *   Canonical host arrays are FP64, complex = [re, im]:
 *     links  [V][4][3][3][2]  (mu = 0:x 1:y 2:z 3:t, row-major colour matrix)
 *     spinor [V][4][3][2]     (spin-major, colour minor), nrhs of them back to back.
 *   Device fields passed to dd_apply_D / dd_sap_smooth are in the library's
 *   internal blocked layout for a given precision; dd_field_bytes gives the
 *   size of one field and dd_pack / dd_unpack convert from / to canonical FP64.
 *
 * Ownership. dd_create_* copy what they need into library-owned device memory;
 *   the caller may free its arrays on return. dd_destroy frees a handle. Device
 *   buffers passed to compute calls are owned by the caller and must stay
 *   valid until the work queued on the given stream has finished.
 *
 * Errors. Every int-returning call returns DD_OK (0) or a negative DD_E* code
 *   and never aborts or traps; dd_last_error() returns a message for the
 *   calling thread's most recent failure.
 *
 * Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream). Compute calls are asynchronous on that stream unless stated.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DD_OK = 0,
  DD_EINVAL = -1,     /* bad argument (null pointer, bad sizes or layout)      */
  DD_ENOMEM = -2,     /* device or host allocation failed                      */
  DD_ECUDA = -3,      /* a CUDA runtime call failed                            */
  DD_ENOTCONV = -4,   /* max_iter reached; x holds the best iterate            */
  DD_ETIMEOUT = -5,   /* a bounded device or host wait expired                 */
  DD_ECANCELLED = -6, /* the request was cancelled                             */
  DD_EBUSY = -7,      /* admission refused (memory budget or slots)            */
  DD_ENOTFOUND = -8   /* unknown ticket                                        */
};

/* storage precisions; arithmetic is FP32 for all but DD_F64 */
enum { DD_F64 = 0, DD_F32 = 1, DD_F16 = 2, DD_BF16 = 3 };
/* Half-precision storage with a per-site scale ("block-float"; the paper's
 * half precision, Sec. 3.1, is plain FP16, the scale is this library's
 * reduced-byte variant of it): spinor fields hold 16-bit fixed-point
 * components q (|q| <= 32767) and per site one FP32 scale n, the largest
 * modulus of its 24 real
 * components, the value being q n / 32767 (q = round-to-nearest-even of
 * v 32767 / n; n = 0 stores zeros); 52 bytes per site, block-major like the
 * other fields (per block 3 chunk rows of 16 bytes x Vb sites, then Vb FP32
 * scales). Operator tiles (links, clover, inverses) are stored as in DD_F16.
 * Accepted wherever DD_F16 is, except by dd_create_mg (DD_EINVAL). */
enum { DD_F16N = 5 };
/* dd_apply_D only (no counterpart in the paper): FP64 input and output
 * fields, double-float arithmetic (pairs of FP32, ~48-bit significands) on
 * the operator's pre-split FP64 links and clover; the operator a
 * mixed-precision dd_solve uses for its true residual. Operators created with
 * a DD_F64 smoother do not hold these fields (DD_EINVAL). A diagnostic path:
 * it allocates one temporary field and synchronises `stream` on return. */
enum { DD_F64_DF = 4 };

/* data location flags for dd_solve / requests */
enum { DD_HOST = 0, DD_DEVICE = 1 };

typedef struct dd_lattice_s *dd_lattice_t;
typedef struct dd_gauge_s *dd_gauge_t;
typedef struct dd_op_s *dd_op_t;
typedef struct dd_server_s *dd_server_t;
typedef struct dd_mg_s *dd_mg_t;

/* Library version string, never NULL. */
const char *dd_version(void);

/* Message of the calling thread's last failure ("" if none). */
const char *dd_last_error(void);

/* Diagnostics: number of CUDA kernels this library has launched so far in
 * this process (all threads). */
uint64_t dd_kernel_launches(void);

/* Diagnostics (no counterpart in the paper): waits for all work on the
 * current device, then returns DD_OK, or DD_ETIMEOUT if any bounded wait
 * inside a kernel (the Schwarz kernel's wait for its staged tiles, about one
 * second of SM clock) has expired since the previous call; a kernel whose
 * wait expired leaves the blocks it had not finished unsmoothed. Clears the
 * count. DD_ECUDA if the device reports an error. */
int dd_device_status(void);

/* Self-test of the kernels' bounded wait (no counterpart in the paper): one
 * CTA stages 16 bytes by a bulk copy and waits on its barrier. expire == 0:
 * the copy completes, DD_OK. expire != 0: the barrier is told to expect more
 * bytes than are copied, the wait expires after about one second, the kernel
 * raises the flag that dd_device_status reports and returns; DD_OK means the
 * expiry was observed and the context is still usable. Synchronous. */
int dd_selftest_wait(int expire);

/* Measurement of the tensor-core question (no counterpart in the paper): the
 * link product of a Schwarz block with a tile of 12 right-hand sides - a
 * 3x3 complex link times 24 complex colour vectors, i.e. a real 6x6 by 6x24
 * product per site and direction - for `ctas` thread blocks of 64
 * site-directions, `reps` times from shared memory. method 0: FP32 operands,
 * FP32 CUDA-core arithmetic; 1: FP16 operands, warp-level tensor-core
 * products (mma.sync m16n8k16, two site-directions block-diagonal in one
 * 16x16 operand, FP32 accumulation); 2: FP16 operands, FP32 CUDA-core
 * arithmetic. *ms receives the time of the `reps` passes (CUDA events, legacy
 * stream); rel_diff (may be NULL) the largest difference of one pass's
 * products from method 0's on the same inputs (exact in FP16), relative to
 * the largest product. Allocates its buffers; synchronous. */
int dd_bench_link_product(int method, int ctas, int reps, double *ms, double *rel_diff);

/* ------------------------------------------------------------------ setup */

/* Lattice geometry and storage tiling. dims {T,Z,Y,X} >= 2 each; block as in
 * Conventions. antiperiodic_t != 0 puts a -1 on fermion hops across the time
 * edge. Returns DD_EINVAL on a bad shape. */
int dd_create_lattice(const int dims[4], const int block[4], int antiperiodic_t, dd_lattice_t *out);

/* Number of sites V and the bytes of one spinor field of precision `prec`. */
long dd_lattice_volume(dd_lattice_t lat);
size_t dd_field_bytes(dd_lattice_t lat, int prec);

/* Gauge field from host links [V][4][3][3][2] (canonical, FP64). Synchronous. */
int dd_create_gauge(dd_lattice_t lat, const double *links_host, dd_gauge_t *out);

/* Wilson-clover operator on `gauge` with clover coefficient c_sw and bare mass
 * m0, for the Schwarz smoother's storage precision `prec` (DD_F64, DD_F32,
 * DD_F16, DD_BF16, DD_F16N). Builds on the device (FP64): the clover term C(n) from the
 * four-leaf plaquette sum, A(n) = 4 + m0 + C(n) as two 6x6 Hermitian chirality
 * blocks per site, and the inverses of the even-site blocks; stores them in
 * FP64 (true residual), FP32 (outer-solver operator) and `prec` (smoother);
 * with prec != DD_F64 also the FP64 links and blocks split into double-float
 * pairs (the true residual of mixed-precision solves).
 * Returns DD_EINVAL if a 6x6 block is singular. Synchronous. */
int dd_create_op(dd_gauge_t gauge, double c_sw, double m0, int prec, dd_op_t *out);

/* Wilson-clover operator on `gauge` with caller-supplied site blocks
 * A(n) = 4 + m0 + C(n) (the clover term computed elsewhere, e.g. by the
 * calling application), host FP64 [V][2][6][6][2] in the layout of
 * dd_op_get_clover (chirality block h = spins {2h, 2h+1}; row/column index
 * 3*(spin - 2h) + colour; canonical site order). Each block's Hermitian
 * part is used. The even-site inverses are formed on the device; storage as
 * for dd_create_op. DD_EINVAL if an even-site block is singular. The caller
 * keeps ownership of clover_host. Synchronous. */
int dd_create_op_clover(dd_gauge_t gauge, const double *clover_host, int prec, dd_op_t *out);

/* Copy the clover site blocks A(n) of `op` (FP64) to host memory as
 * [V][2][6][6][2] (chirality block h = spins {2h, 2h+1}; row/column index
 * 3*(spin - 2h) + colour), canonical site order. Synchronous. */
int dd_op_get_clover(dd_op_t op, double *host_out);

/* Free any handle returned by this library (lattice, gauge, op, server).
 * Destroying a lattice or gauge still used by an op is deferred until the op
 * is destroyed. NULL is ignored. */
void dd_destroy(void *handle);

/* ----------------------------------------------------------- layouts */

/* Canonical FP64 spinors (device memory, [nrhs][V][4][3][2]) -> internal
 * layout of precision `prec`, each value multiplied by `scale`, rounded to
 * nearest even. Asynchronous on `stream`. */
int dd_pack(dd_lattice_t lat, int prec, const double *canon_dev, void *field_dev, int nrhs,
            double scale, void *stream);

/* Internal layout of precision `prec` -> canonical FP64 (device memory),
 * multiplied by `scale`. Asynchronous on `stream`. */
int dd_unpack(dd_lattice_t lat, int prec, const void *field_dev, double *canon_dev, int nrhs,
              double scale, void *stream);

/* ------------------------------------------------------------ compute */

/* out = D in for nrhs fields (internal layout, precision `prec`, field r at
 * byte offset r * dd_field_bytes). `prec` must be DD_F64, DD_F32 or the op's
 * smoother precision. in and out must not overlap. Asynchronous. */
int dd_apply_D(dd_op_t op, int prec, const void *in_dev, void *out_dev, int nrhs, void *stream);

typedef struct {
  int sweeps;     /* Schwarz sweeps (each = colour 0 then colour 1), >= 1        */
  int mr_steps;   /* MR steps per block solve, >= 0                              */
  int x_is_zero;  /* 1: x is not read and taken as 0 (preconditioner use)        */
  int rhs_tile;   /* right-hand sides sharing one staged block (0 = autotuned)   */
} dd_sap_params;

/* Schwarz alternating procedure in the op's smoother precision: x is updated
 * by `sweeps` red-black sweeps for the system D x = b, each block solved by
 * even-odd MR (Sec. 3.1, Tables 1-2). b and x: nrhs internal-layout fields of
 * that precision. Asynchronous. */
int dd_sap_smooth(dd_op_t op, const dd_sap_params *p, const void *b_dev, void *x_dev, int nrhs,
                  void *stream);

/* The Schwarz smoother of dd_sap_smooth for right-hand sides of several
 * operators at once - on lattices of different sizes too - in one launch per
 * colour phase (the batched form of Sec. 3.1's Schwarz method): operator k
 * smooths nrhs[k] fields, contiguous from b[k] and x[k] (internal layout of
 * its smoother precision). All operators need the same smoother precision
 * and Schwarz block shape; 1 <= nops <= 8 and at most 64 right-hand sides in
 * all (DD_EINVAL otherwise). Each right-hand side's result is the one
 * dd_sap_smooth gives it. Asynchronous on `stream` (its work fields are
 * stream-ordered allocations). */
int dd_sap_smooth_multi(int nops, const dd_op_t *ops, const int *nrhs, const dd_sap_params *p,
                        const void *const *b_dev, void *const *x_dev, void *stream);

typedef struct {
  double tol;           /* target true relative residual ||b - D x|| / ||b||        */
  int restart;          /* FGMRES restart length m (1..64)                          */
  int max_iter;         /* cap on preconditioned Arnoldi steps per right-hand side  */
  dd_sap_params sap;    /* smoother applied once per Arnoldi step                   */
  double inner_reduction; /* a cycle stops once its estimate fell by this factor
                             (0: run to tol; mixed precision uses ~1e-5)            */
  int where;            /* DD_HOST or DD_DEVICE for b and x                          */
  int use_x0;           /* 1: x holds the initial guess; 0: start from x = 0         */
  dd_mg_t mg;           /* NULL: precondition with `sap`; else the two-level
                           preconditioner of dd_create_mg (same operator)          */
  int outer_f64;        /* 1: with a mixed-precision op, keep the Krylov basis and
                           the true residual's Dslash in IEEE FP64 too, instead of
                           double-float (slower on GB300: its FP64 rate is a small
                           fraction of FP32); not with `mg`. 0: the default        */
} dd_solve_params;

typedef struct {
  int status;             /* DD_OK, DD_ENOTCONV, ...                               */
  int iterations;         /* preconditioned Arnoldi steps                          */
  int cycles;             /* restart cycles                                        */
  double true_rel_residual; /* ||b - D x|| / ||b|| recomputed at exit (see dd_solve) */
  double est_rel_residual;  /* FGMRES estimate at exit                              */
  double ms_total, ms_sap, ms_dirac, ms_orth; /* wall time split (ms)               */
} dd_solve_info;

/* Solve D x = b for nrhs canonical FP64 right-hand sides ([nrhs][V][4][3][2],
 * host or device per p->where) with SAP-preconditioned FGMRES. The smoother
 * runs in the op's precision. With an FP64 op the orthogonalisation, the
 * least-squares update and the true residual are IEEE FP64; with a
 * mixed-precision op the Krylov basis and the true residual's Dslash use
 * double-float arithmetic (FP32 pairs, ~48-bit significands) unless
 * p->outer_f64 asks for IEEE FP64, the least-squares update, x and the
 * residual norms stay FP64. x receives the solutions
 * (and holds the initial guesses if p->use_x0). info (may be NULL) receives
 * nrhs records. Returns DD_OK when every right-hand side converged, else
 * DD_ENOTCONV (x holds the best iterates) or an error. Synchronous with
 * respect to the host; work runs on `stream`. */
int dd_solve(dd_op_t op, const dd_solve_params *p, const double *b, double *x, int nrhs,
             dd_solve_info *info, void *stream);

/* The workspace of dd_solve (Krylov basis, preconditioned vectors, scratch
 * fields and reduction buffers: about 6 kB per site and right-hand side at
 * restart 16) is cached when the call ends and reused by the next dd_solve
 * that needs buffers of the same sizes on the same device, which saves the
 * allocation and release (milliseconds, and a device synchronisation) per
 * call. A solve that cannot allocate releases the cache first; the cache
 * holds at most half of the device memory and 64 MB of pinned host memory;
 * dd_server_create releases it (the server budgets device memory itself and
 * its workers free their buffers). This call frees every cached buffer (all
 * devices), e.g. to return the memory to other users. Returns DD_OK. */
int dd_release_workspace(void);

/* ------------------------------------------------------- two-level multigrid */

typedef struct {
  int n_vectors;        /* test vectors N (1..32); coarse sites carry 2N unknowns          */
  int setup_iters;      /* smoother applications to each test vector before P is formed    */
  int coarse_max_iter;  /* coarse GMRES steps per application (1..64, one cycle from 0)    */
  double coarse_tol;    /* coarse GMRES stops once its residual estimate falls by this     */
  dd_sap_params smoother; /* Schwarz post-smoother (and the setup's smoother)              */
} dd_mg_params;

/* Two-level preconditioner of the paper's DD-alpha-AMG (Sec. 1; its
 * fine-level smoother is the Schwarz method of Sec. 3.1): aggregates are the
 * lattice's Schwarz blocks; the test vectors (host, N canonical FP64 spinor
 * fields [N][V][4][3][2], e.g. seeded random fields) are each smoothed by
 * `setup_iters` Schwarz applications, then orthonormalised per aggregate and
 * chirality (spins {0,1} / {2,3}) by modified Gram-Schmidt in vector order to
 * form the interpolation P; the coarse operator is D_c = P^dagger D P (FP32,
 * nearest-neighbour stencil on the block grid with 2N x 2N blocks). One
 * application is M r = P e_c + SAP(r - D P e_c) with e_c from GMRES on D_c.
 * Synchronous; the object keeps a reference on `op`. Blocks of at most 256
 * sites. */
int dd_create_mg(dd_op_t op, const dd_mg_params *p, const double *test_vectors_host, dd_mg_t *out);

/* Coarse vectors are [aggregate][chirality h][k] complex FP32 (2 floats),
 * aggregates in block order (x fastest); dd_mg_coarse_length gives their
 * number of complex entries. Fine fields are FP32 internal-layout fields. The
 * calls below use the object's own workspace: one stream at a time.
 * Asynchronous on `stream`. */
size_t dd_mg_coarse_length(dd_mg_t mg);
int dd_mg_restrict(dd_mg_t mg, const void *fine_f32, void *coarse, void *stream);   /* P^dagger r */
int dd_mg_prolong(dd_mg_t mg, const void *coarse, void *fine_f32, void *stream);    /* P c */
int dd_mg_coarse_apply(dd_mg_t mg, const void *coarse_in, void *coarse_out, void *stream); /* D_c c */
int dd_mg_precondition(dd_mg_t mg, const void *r_f32, void *x_f32, void *stream);   /* x = M r */

/* Size of the fixed device scratch array behind dd_solve_noalloc: 64 MiB. */
#define DD_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Solve D x = b for ONE right-hand side without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device (or pinned host) memory at solve time - for example
 * code running where cudaMalloc is forbidden or would disturb a fixed memory
 * plan. It runs the same SAP-preconditioned FGMRES as dd_solve, with the
 * whole workspace taken from one file-scope device array of
 * DD_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * process exit. b_dev and x_dev are canonical FP64 spinors in DEVICE memory
 * ([V][4][3][2]); x_dev receives the solution (and holds the initial guess if
 * p->use_x0; p->where is ignored). info may be NULL.
 * Limits and rules: returns DD_EINVAL, before doing any work, when the
 * lattice and restart length need more scratch than the array holds (about
 * 6 kB per site at restart 16 with an FP32 smoother, so lattices up to
 * roughly 10^4 sites); all calls in the process share the array, so calls
 * whose GPU work overlaps (other streams, threads or concurrent calls) race
 * and must be serialised by the caller; the array keeps the previous call's
 * contents, and each call clears what it needs zeroed itself. The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream capture
 * on the device, and do not call this entry point on a device after
 * cudaDeviceReset in the same process (the address is kept). Nothing is
 * tuned or captured inside the call: every kernel runs in the launch variant
 * the autotuner already chose for this lattice and precision (e.g. by an
 * earlier dd_solve of the same shape, or a DD_TUNE_CACHE file), else in its
 * default variant, and the smoother's launches are enqueued one by one. The
 * host side uses about 72 KB of the calling thread's stack. Synchronous with
 * respect to the host; work runs on `stream`. */
int dd_solve_noalloc(dd_op_t op, const dd_solve_params *p, const double *b_dev, double *x_dev,
                     dd_solve_info *info, void *stream);

/* ------------------------------------------------------------ serving */

typedef struct {
  size_t hbm_budget_bytes; /* device bytes the server may hold for requests (0 = 80% of free) */
  int max_slots;           /* requests on the device at once (1..64)                 */
  int max_batch_rhs;       /* right-hand sides batched per solve launch (1..64)       */
} dd_server_params;

typedef struct {
  dd_op_t op;             /* resident operator the request solves with                  */
  const double *b_host;   /* nrhs canonical FP64 right-hand sides (copied on submit)     */
  int nrhs;
  dd_solve_params params; /* `where` is ignored: requests are host-to-host               */
} dd_request;

enum { DD_QUEUED = 0, DD_RUNNING = 1, DD_DONE = 2, DD_FAILED = 3, DD_CANCELLED_STATE = 4 };

/* Start a server: a host scheduler thread that admits requests while device
 * memory and slots allow, batches right-hand sides of the same operator, runs
 * batches on separate streams so they overlap, and retires each right-hand
 * side as it converges. */
int dd_server_create(const dd_server_params *p, dd_server_t *out);

/* Queue a request (b is copied). *ticket identifies it. DD_EBUSY if the
 * request alone can never fit the memory budget. The server does not take a
 * reference on req->op (or on params.mg): keep them alive until the request
 * has reached a final state (DONE, FAILED or CANCELLED, seen by dd_poll) or
 * the server has been destroyed. */
int dd_submit(dd_server_t s, const dd_request *req, uint64_t *ticket);

/* State of a ticket. When DONE, x_out (may be NULL) receives nrhs canonical
 * solutions and info (may be NULL) nrhs records; the ticket is then released.
 * Times in info are measured from submission. */
int dd_poll(dd_server_t s, uint64_t ticket, int *state, double *x_out, dd_solve_info *info);

/* Cancel a queued or running request (its work stops at the next step). */
int dd_cancel(dd_server_t s, uint64_t ticket);

typedef struct {
  uint64_t submitted, completed, failed, cancelled;
  double p50_ms, p99_ms;    /* latency from submit to done, completed requests */
  double rhs_per_s;         /* completed right-hand sides per second of server time */
  size_t bytes_in_use;      /* device bytes held by admitted requests */
} dd_server_stats;

int dd_server_get_stats(dd_server_t s, dd_server_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
