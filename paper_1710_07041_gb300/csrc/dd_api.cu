// C ABI: handles, set-up (the "data-layout transformations at solver entry"
// of Sec. 5 happen in dd_create_* and dd_pack), and the compute entry points.
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "dd_internal.cuh"

namespace dd {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

int cuda_fail(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return DD_OK;
  set_error("%s: %s", where, cudaGetErrorString(e));
  return DD_ECUDA;
}

static std::atomic<unsigned long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

int launched(const char *where) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cuda_fail(cudaGetLastError(), where);
}

enum : int { MAGIC_LAT = 0x4c415431, MAGIC_GAUGE = 0x47415531, MAGIC_OP = 0x4f505231, MAGIC_SERVER = 0x53525631,
             MAGIC_MG = 0x4d475231 };

static bool pow2(int v) { return v >= 2 && (v & (v - 1)) == 0; }
static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) l++;
  return l;
}

const OpFields *fields_for(const Op *op, int prec) {
  if (prec == DD_F64) return &op->f64;
  if (prec == DD_F32) return &op->f32;
  if (prec == op->prec) return &op->fp;
  return nullptr;
}

static void free_fields(OpFields &f) {
  if (f.links_full != f.links) cudaFree(f.links_full);
  cudaFree(f.links);
  cudaFree(f.clov);
  cudaFree(f.cinv);
  f = OpFields{};
}

static void release_lattice(Lattice *l) {
  if (l && --l->refs == 0) {
    l->magic = 0;
    delete l;
  }
}
static void release_gauge(Gauge *g) {
  if (g && --g->refs == 0) {
    cudaFree(g->links_canon);
    release_lattice(g->lat);
    g->magic = 0;
    delete g;
  }
}

void release_op(Op *op) {
  if (!op || --op->refs > 0) return;
  free_fields(op->f64);
  free_fields(op->f32);
  if (half_tiles(op->prec)) free_fields(op->fp);
  free_fields(op->fdf);
  release_gauge(op->gauge);
  op->magic = 0;
  delete op;
}

// checked-build counters of all translation units
static std::vector<unsigned (*)()> &bounds_readers() {
  static std::vector<unsigned (*)()> v;
  return v;
}
int register_bounds_reader(unsigned (*read)()) {
  bounds_readers().push_back(read);
  return 1;
}
unsigned bounds_errors_all() {
  unsigned n = 0;
  for (auto r : bounds_readers()) n += r();
  return n;
}

void destroy_server(void *s);  // dd_server.cu
void destroy_mg(void *h);      // dd_mg.cu
int server_magic_ok(void *s);

}  // namespace dd

using namespace dd;

extern "C" {

const char *dd_version(void) { return "dd-gb300 0.1 (sm_103a)"; }

const char *dd_last_error(void) { return g_err.c_str(); }

uint64_t dd_kernel_launches(void) { return g_launches.load(); }

int dd_device_status(void) { return device_wait_status(); }

int dd_selftest_wait(int expire) { return wait_selftest(expire); }

int dd_create_lattice(const int dims[4], const int block[4], int antiperiodic_t, dd_lattice_t *out) {
  if (!dims || !block || !out) {
    set_error("dd_create_lattice: null argument");
    return DD_EINVAL;
  }
  Geom g{};
  long long V = 1;
  for (int mu = 0; mu < 4; mu++) {
    int L = dims[3 - mu], B = block[3 - mu];
    if (L < 2 || !pow2(B) || L % B != 0 || (L / B) % 2 != 0) {
      set_error("dd_create_lattice: direction %d: extent %d, block %d (block must be a power of two >= 2 "
                "dividing the extent an even number of times)", mu, L, B);
      return DD_EINVAL;
    }
    g.L[mu] = L;
    g.bd[mu] = B;
    g.lbd[mu] = ilog2(B);
    g.nb[mu] = L / B;
    V *= L;
  }
  g.bstride[0] = 1;
  for (int mu = 1; mu < 4; mu++) g.bstride[mu] = g.bstride[mu - 1] * g.nb[mu - 1];
  g.Vb = g.bd[0] * g.bd[1] * g.bd[2] * g.bd[3];
  g.Vh = g.Vb / 2;
  g.nblocks = (int)(V / g.Vb);
  g.V = V;
  g.antiperiodic = antiperiodic_t ? 1 : 0;
  Lattice *l = new (std::nothrow) Lattice;
  if (!l) return DD_ENOMEM;
  l->magic = MAGIC_LAT;
  l->g = g;
  memcpy(l->dims, dims, sizeof l->dims);
  memcpy(l->block, block, sizeof l->block);
  l->refs = 1;
  *out = (dd_lattice_t)l;
  return DD_OK;
}

long dd_lattice_volume(dd_lattice_t lat) {
  Lattice *l = (Lattice *)lat;
  return (l && l->magic == MAGIC_LAT) ? (long)l->g.V : -1;
}

size_t dd_field_bytes(dd_lattice_t lat, int prec) {
  Lattice *l = (Lattice *)lat;
  if (!l || l->magic != MAGIC_LAT || !storage_prec(prec)) return 0;
  return (size_t)l->g.V * spinor_site_bytes(prec);
}

int dd_create_gauge(dd_lattice_t lat, const double *links, dd_gauge_t *out) {
  Lattice *l = (Lattice *)lat;
  if (!l || l->magic != MAGIC_LAT || !links || !out) {
    set_error("dd_create_gauge: bad argument");
    return DD_EINVAL;
  }
  Gauge *g = new (std::nothrow) Gauge;
  if (!g) return DD_ENOMEM;
  size_t bytes = (size_t)l->g.V * 72 * sizeof(double);
  if (cudaMalloc(&g->links_canon, bytes) != cudaSuccess) {
    delete g;
    set_error("dd_create_gauge: out of device memory (%zu bytes)", bytes);
    return DD_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(g->links_canon, links, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(g->links_canon);
    delete g;
    return cuda_fail(e, "dd_create_gauge: copy");
  }
  g->magic = MAGIC_GAUGE;
  g->lat = l;
  l->refs++;
  g->refs = 1;
  *out = (dd_gauge_t)g;
  return DD_OK;
}

static int alloc_fields(const Geom &g, int prec, OpFields &f) {
  f.prec = prec;
  size_t pb = pair_bytes(prec);
  if (cudaMalloc(&f.links, (size_t)g.V * 4 * link_pairs_of(prec) * pb) != cudaSuccess ||
      (link_pairs_of(prec) != 9 && cudaMalloc(&f.links_full, (size_t)g.V * 36 * pb) != cudaSuccess) ||
      cudaMalloc(&f.clov, (size_t)g.V * 36 * pb) != cudaSuccess ||
      cudaMalloc(&f.cinv, (size_t)g.V / 2 * 36 * pb) != cudaSuccess) {
    free_fields(f);
    set_error("dd_create_op: out of device memory");
    return DD_ENOMEM;
  }
  if (link_pairs_of(prec) == 9) f.links_full = f.links;
  return DD_OK;
}

}  // extern "C"

// Shared tail of the two operator constructors: `fill` writes the FP64 site
// blocks and even-site inverses (and may flag a singular block in *bad); the
// links and the lower-precision copies follow.
template <typename Fill>
static int create_op(Gauge *ga, double c_sw, double m0, int prec, Fill fill, dd_op_t *out) {
  const Geom &g = ga->lat->g;
  Op *op = new (std::nothrow) Op;
  if (!op) return DD_ENOMEM;
  op->magic = MAGIC_OP;
  op->gauge = ga;
  op->lat = ga->lat;
  op->c_sw = c_sw;
  op->m0 = m0;
  op->prec = prec;
  int rc = alloc_fields(g, DD_F64, op->f64);
  if (rc == DD_OK) rc = alloc_fields(g, DD_F32, op->f32);
  if (rc == DD_OK && half_tiles(prec)) rc = alloc_fields(g, prec, op->fp);
  int *bad = nullptr;
  if (rc == DD_OK && cudaMalloc(&bad, sizeof(int)) != cudaSuccess) rc = DD_ENOMEM;
  cudaStream_t st = 0;
  if (rc == DD_OK) rc = cuda_fail(cudaMemsetAsync(bad, 0, sizeof(int), st), "memset");
  if (rc == DD_OK) rc = fill(g, (double *)op->f64.clov, (double *)op->f64.cinv, bad, st);
  if (rc == DD_OK) rc = launch_pack_links(g, DD_F64, ga->links_canon, op->f64.links, bad, st);
  if (rc == DD_OK) rc = launch_pack_links(g, DD_F32, ga->links_canon, op->f32.links, bad, st);
  if (rc == DD_OK) rc = launch_pack_links_full(g, DD_F32, ga->links_canon, op->f32.links_full, st);
  if (rc == DD_OK) rc = launch_convert_clover(DD_F32, (const double *)op->f64.clov, op->f32.clov, g.nblocks, g.Vb, st);
  if (rc == DD_OK) rc = launch_convert_clover(DD_F32, (const double *)op->f64.cinv, op->f32.cinv, g.nblocks, g.Vh, st);
  if (rc == DD_OK && half_tiles(prec)) {
    rc = launch_pack_links(g, prec, ga->links_canon, op->fp.links, bad, st);
    if (rc == DD_OK) rc = launch_pack_links_full(g, prec, ga->links_canon, op->fp.links_full, st);
    if (rc == DD_OK) rc = launch_convert_clover(prec, (const double *)op->f64.clov, op->fp.clov, g.nblocks, g.Vb, st);
    if (rc == DD_OK) rc = launch_convert_clover(prec, (const double *)op->f64.cinv, op->fp.cinv, g.nblocks, g.Vh, st);
  }
  if (rc == DD_OK && prec != DD_F64) {
    // double-float copies of the FP64 links and site blocks (the true residual of mixed-precision solves)
    op->fdf.prec = DD_PREC_DF;
    const size_t np = (size_t)g.V * 36;
    if (cudaMalloc(&op->fdf.links, np * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&op->fdf.clov, np * sizeof(float4)) != cudaSuccess) {
      cudaGetLastError();
      set_error("dd_create_op: out of device memory");
      rc = DD_ENOMEM;
    }
    if (rc == DD_OK) rc = launch_split_pairs((const double *)op->f64.links, op->fdf.links, np, st);
    if (rc == DD_OK) rc = launch_split_pairs((const double *)op->f64.clov, op->fdf.clov, np, st);
  }
  int hbad = 0;
  if (rc == DD_OK) rc = cuda_fail(cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost), "dd_create_op");
  cudaFree(bad);
  if (rc == DD_OK && (hbad & 1)) {
    set_error("dd_create_op: an even-site clover block A = 4 + m0 + C is singular");
    rc = DD_EINVAL;
  } else if (rc == DD_OK && (hbad & 2)) {
    set_error("dd_create_op: a link is not special unitary (row 2 differs from conj(row0 x row1) by more than "
              "1e-6); the 32- and 16-bit operator fields store two rows per link");
    rc = DD_EINVAL;
  }
  if (rc != DD_OK) {
    free_fields(op->f64);
    free_fields(op->f32);
    free_fields(op->fp);
    free_fields(op->fdf);
    delete op;
    return rc;
  }
  if (prec == DD_F64) op->fp = op->f64;
  if (prec == DD_F32) op->fp = op->f32;
  op->refs = 1;
  ga->refs++;
  *out = (dd_op_t)op;
  return DD_OK;
}

extern "C" {

int dd_create_op(dd_gauge_t gauge, double c_sw, double m0, int prec, dd_op_t *out) {
  Gauge *ga = (Gauge *)gauge;
  if (!ga || ga->magic != MAGIC_GAUGE || !out || !storage_prec(prec) || !std::isfinite(c_sw) ||
      !std::isfinite(m0)) {
    set_error("dd_create_op: bad argument");
    return DD_EINVAL;
  }
  return create_op(
      ga, c_sw, m0, prec,
      [&](const Geom &g, double *clov, double *cinv, int *bad, cudaStream_t st) {
        return launch_build_clover(g, ga->links_canon, c_sw, m0, clov, cinv, bad, st);
      },
      out);
}

int dd_create_op_clover(dd_gauge_t gauge, const double *clover_host, int prec, dd_op_t *out) {
  Gauge *ga = (Gauge *)gauge;
  if (!ga || ga->magic != MAGIC_GAUGE || !clover_host || !out || !storage_prec(prec)) {
    set_error("dd_create_op_clover: bad argument");
    return DD_EINVAL;
  }
  const size_t bytes = (size_t)ga->lat->g.V * 144 * sizeof(double);
  double *dev = nullptr;
  if (cudaMalloc(&dev, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("dd_create_op_clover: out of device memory (%zu bytes)", bytes);
    return DD_ENOMEM;
  }
  int rc = cuda_fail(cudaMemcpy(dev, clover_host, bytes, cudaMemcpyHostToDevice), "dd_create_op_clover: copy");
  if (rc == DD_OK)
    rc = create_op(
        ga, NAN, NAN, prec,
        [&](const Geom &g, double *clov, double *cinv, int *bad, cudaStream_t st) {
          return launch_load_clover(g, dev, clov, cinv, bad, st);
        },
        out);
  cudaFree(dev);
  return rc;
}

int dd_op_get_clover(dd_op_t opp, double *host_out) {
  Op *op = (Op *)opp;
  if (!op || op->magic != MAGIC_OP || !host_out) {
    set_error("dd_op_get_clover: bad argument");
    return DD_EINVAL;
  }
  const Geom &g = op->lat->g;
  std::vector<double> tile((size_t)g.V * 72);
  int rc = cuda_fail(cudaMemcpy(tile.data(), op->f64.clov, tile.size() * sizeof(double), cudaMemcpyDeviceToHost),
                     "dd_op_get_clover");
  if (rc) return rc;
  for (int b = 0; b < g.nblocks; b++)
    for (int s = 0; s < g.Vb; s++) {
      long long n = canonical_index(g, b, s);
      for (int h = 0; h < 2; h++) {
        auto pr = [&](int i) {
          size_t idx = (((size_t)b * 36 + 18 * h + i) * g.Vb + s) * 2;
          return std::complex<double>(tile[idx], tile[idx + 1]);
        };
        double *dst = host_out + ((size_t)n * 2 + h) * 72;
        double dg[6] = {pr(0).real(), pr(0).imag(), pr(1).real(), pr(1).imag(), pr(2).real(), pr(2).imag()};
        for (int i = 0; i < 6; i++)
          for (int j = 0; j < 6; j++) {
            std::complex<double> v;
            if (i == j) v = dg[i];
            else if (i < j) v = pr(herm_off(i, j));
            else v = std::conj(pr(herm_off(j, i)));
            dst[(i * 6 + j) * 2] = v.real();
            dst[(i * 6 + j) * 2 + 1] = v.imag();
          }
      }
    }
  return DD_OK;
}

void dd_destroy(void *h) {
  if (!h) return;
  int m = *(int *)h;
  if (m == MAGIC_LAT) {
    release_lattice((Lattice *)h);
  } else if (m == MAGIC_GAUGE) {
    release_gauge((Gauge *)h);
  } else if (m == MAGIC_OP) {
    release_op((Op *)h);
  } else if (m == MAGIC_SERVER) {
    destroy_server(h);
  } else if (m == MAGIC_MG) {
    destroy_mg(h);
  }
}

int dd_pack(dd_lattice_t lat, int prec, const double *canon, void *field, int nrhs, double scale, void *stream) {
  Lattice *l = (Lattice *)lat;
  if (!l || l->magic != MAGIC_LAT || !canon || !field || nrhs < 1 || !storage_prec(prec)) {
    set_error("dd_pack: bad argument");
    return DD_EINVAL;
  }
  return launch_pack(l->g, prec, canon, field, nrhs, scale, (cudaStream_t)stream);
}

int dd_unpack(dd_lattice_t lat, int prec, const void *field, double *canon, int nrhs, double scale, void *stream) {
  Lattice *l = (Lattice *)lat;
  if (!l || l->magic != MAGIC_LAT || !canon || !field || nrhs < 1 || !storage_prec(prec)) {
    set_error("dd_unpack: bad argument");
    return DD_EINVAL;
  }
  return launch_unpack(l->g, prec, field, canon, nrhs, scale, (cudaStream_t)stream);
}

int dd_apply_D(dd_op_t opp, int prec, const void *in, void *out, int nrhs, void *stream) {
  Op *op = (Op *)opp;
  if (!op || op->magic != MAGIC_OP || !in || !out || in == out || nrhs < 1) {
    set_error("dd_apply_D: bad argument");
    return DD_EINVAL;
  }
  if (prec == DD_F64_DF) {
    if (!op->fdf.links) {
      set_error("dd_apply_D: this operator holds no double-float fields (FP64 smoother)");
      return DD_EINVAL;
    }
    const Geom &g = op->lat->g;
    const size_t fb = (size_t)g.V * 24 * 8, n = (size_t)g.V * 12;
    void *tmp = nullptr;   // the split input, one right-hand side at a time
    DD_CUDA(cudaMalloc(&tmp, fb));
    int rc = DD_OK;
    for (int r = 0; r < nrhs && rc == DD_OK; r++) {
      rc = launch_split_pairs((const double *)((const char *)in + r * fb), tmp, n, (cudaStream_t)stream);
      if (rc == DD_OK) rc = launch_dirac_df(g, op->fdf, contiguous(tmp, (char *)out + r * fb, 1, fb), (cudaStream_t)stream);
    }
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaFree(tmp);
    return rc;
  }
  const OpFields *f = fields_for(op, prec);
  if (!f) {
    set_error("dd_apply_D: precision %d not held by this operator", prec);
    return DD_EINVAL;
  }
  return launch_dirac(op->lat->g, *f, in, out, nrhs, (cudaStream_t)stream);
}

int dd_sap_smooth(dd_op_t opp, const dd_sap_params *p, const void *b, void *x, int nrhs, void *stream) {
  Op *op = (Op *)opp;
  if (!op || op->magic != MAGIC_OP || !p || !b || !x || b == x || nrhs < 1 || p->sweeps < 1 || p->mr_steps < 0) {
    set_error("dd_sap_smooth: bad argument");
    return DD_EINVAL;
  }
  // work fields of the incremental colour residual, stream-ordered (without
  // them, e.g. when this allocation fails, every phase forms b - D x)
  cudaStream_t st = (cudaStream_t)stream;
  const Geom &g = op->lat->g;
  const size_t fb = (size_t)g.V * spinor_site_bytes(op->fp.prec);
  void *aux = nullptr;
  if (cudaMallocAsync(&aux, 2 * (size_t)nrhs * fb, st) != cudaSuccess) {
    cudaGetLastError();
    aux = nullptr;
  }
  int rc = launch_sap(g, op->fp, *p, b, x, nrhs, st, aux);
  if (aux) cudaFreeAsync(aux, st);
  return rc;
}

int dd_sap_smooth_multi(int nops, const dd_op_t *ops, const int *nrhs, const dd_sap_params *p,
                        const void *const *b, void *const *x, void *stream) {
  if (nops < 1 || nops > MAX_SAP_GROUPS || !ops || !nrhs || !p || !b || !x || p->sweeps < 1 || p->mr_steps < 0) {
    set_error("dd_sap_smooth_multi: bad argument (1 <= nops <= %d)", MAX_SAP_GROUPS);
    return DD_EINVAL;
  }
  SapLattice lats[MAX_SAP_GROUPS];
  RhsPtrs rp;
  rp.n = 0;
  size_t aux_bytes = 0;
  for (int k = 0; k < nops; k++) {
    const Op *op = (const Op *)ops[k];
    if (!op || op->magic != MAGIC_OP || nrhs[k] < 1 || !b[k] || !x[k] || b[k] == x[k] ||
        rp.n + nrhs[k] > MAX_RHS) {
      set_error("dd_sap_smooth_multi: bad operator %d or right-hand sides (at most %d in all)", k, MAX_RHS);
      return DD_EINVAL;
    }
    const size_t fb = (size_t)op->lat->g.V * spinor_site_bytes(op->fp.prec);
    for (int r = 0; r < nrhs[k]; r++, rp.n++) {
      rp.in[rp.n] = (const char *)b[k] + r * fb;
      rp.out[rp.n] = (char *)x[k] + r * fb;
    }
    lats[k] = SapLattice{op->lat->g, op->fp, nrhs[k]};
    aux_bytes += 2 * (size_t)nrhs[k] * fb;
  }
  // work fields of the incremental colour residual, stream-ordered
  cudaStream_t st = (cudaStream_t)stream;
  char *aux = nullptr;
  if (cudaMallocAsync((void **)&aux, aux_bytes, st) != cudaSuccess) {
    cudaGetLastError();
    aux = nullptr;
  }
  AuxPtrs ax{};
  for (int k = 0, i = 0; aux && k < nops; k++) {
    const size_t fb = (size_t)lats[k].g.V * spinor_site_bytes(lats[k].f.prec);
    for (int r = 0; r < nrhs[k]; r++, i++) {
      ax.e[i] = aux;
      ax.r[i] = aux + fb;
      aux += 2 * fb;
    }
  }
  int rc = launch_sap_lattices(lats, nops, *p, rp, st, ax.e[0] ? &ax : nullptr);
  if (ax.e[0]) cudaFreeAsync(ax.e[0], st);
  return rc;
}

}  // extern "C"
