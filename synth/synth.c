/*
 * Seeded synthetic inputs for the Wilson-clover SAP-FGMRES path.
 *
 * This module only PREPARES inputs: gauge links, random right-hand sides and
 * random gauge transformations. It holds none of the solver's arithmetic (no
 * Dirac operator, no clover term, no Schwarz or Krylov step). Both the FP64
 * oracle and the GPU path receive what it writes as plain host arrays.
 *
 * The paper's gauge ensembles (Sec. 4, 16^3x32 and 32^3x96 lattices produced
 * with Chroma/QDP++) are not available, so links are synthetic:
 *   U = exp(i * eps * H),  H = sum_a w_a lambda_a / 2,  w_a ~ N(0,1),
 * with lambda_a the eight Gell-Mann matrices, optionally followed by isotropic
 * stout smearing (Morningstar and Peardon, Phys. Rev. D 69 (2004) 054501):
 *   C = rho * sum_{nu != mu} (upper staple + lower staple),
 *   Omega = C U^dagger,
 *   Q = (i/2)(Omega^dagger - Omega) - (i/6) tr(Omega^dagger - Omega),
 *   U' = exp(i Q) U,  all links updated simultaneously.
 *
 * Random numbers come from a counter-based generator: the 64-bit value for
 * counter c under seed s is splitmix64 (Steele, Lea and Flood, OOPSLA 2014)
 * applied to s * 0x9E3779B97F4A7C15 + c; normal deviates use the Box-Muller
 * transform. Every value depends only on (seed, counter), so results do not
 * depend on the thread count.
 *
 * Layouts (all double precision, complex as [re, im]):
 *   lattice dims  d[4] = {T, Z, Y, X}; site n = x + X*(y + Y*(z + Z*t))
 *   directions    mu = 0:x, 1:y, 2:z, 3:t
 *   links         [V][4][3][3][2]   (row-major colour matrix per direction)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

static inline uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* uniform in (0, 1]: top 53 bits of the hash, shifted off zero */
static inline double unif(uint64_t seed, uint64_t ctr) {
  uint64_t v = sm64(seed * 0x9E3779B97F4A7C15ULL + ctr);
  return ((double)(v >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

/* standard normal deviate number k of stream (seed, base): Box-Muller on the
 * uniform pair (2k, 2k+1) of that stream */
static inline double gauss(uint64_t seed, uint64_t ctr) {
  const double two_pi = 6.283185307179586476925286766559;
  double u1 = unif(seed, 2 * ctr), u2 = unif(seed, 2 * ctr + 1);
  return sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
}

static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}

/* 3x3 complex helpers, row-major m[r*3+c] */
static void mm(const cplx *a, const cplx *b, cplx *o) {
  cplx t[9];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) {
      cplx s = {0, 0};
      for (int k = 0; k < 3; k++) {
        cplx p = cmul(a[r * 3 + k], b[k * 3 + c]);
        s.re += p.re; s.im += p.im;
      }
      t[r * 3 + c] = s;
    }
  memcpy(o, t, sizeof t);
}
static void dag(const cplx *a, cplx *o) {
  cplx t[9];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) { t[r * 3 + c].re = a[c * 3 + r].re; t[r * 3 + c].im = -a[c * 3 + r].im; }
  memcpy(o, t, sizeof t);
}
/* a * b^dagger */
static void mmd(const cplx *a, const cplx *b, cplx *o) { cplx t[9]; dag(b, t); mm(a, t, o); }
/* a^dagger * b */
static void mdm(const cplx *a, const cplx *b, cplx *o) { cplx t[9]; dag(a, t); mm(t, b, o); }

/* exp(X) for a 3x3 complex X by scaling and squaring with a Taylor series.
 * Terms are added until they fall below 1e-18 of the running sum. */
static void expm3(const cplx *x, cplx *out) {
  double nrm = 0;
  for (int i = 0; i < 9; i++) nrm += x[i].re * x[i].re + x[i].im * x[i].im;
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.25) { nrm *= 0.5; s++; }
  double sc = ldexp(1.0, -s);
  cplx y[9], term[9], sum[9];
  for (int i = 0; i < 9; i++) { y[i].re = x[i].re * sc; y[i].im = x[i].im * sc; }
  for (int i = 0; i < 9; i++) { sum[i].re = (i % 4 == 0); sum[i].im = 0; term[i] = sum[i]; }
  for (int k = 1; k < 40; k++) {
    mm(term, y, term);
    double tn = 0;
    for (int i = 0; i < 9; i++) {
      term[i].re /= k; term[i].im /= k;
      sum[i].re += term[i].re; sum[i].im += term[i].im;
      tn += term[i].re * term[i].re + term[i].im * term[i].im;
    }
    if (tn < 1e-36) break;
  }
  for (int i = 0; i < s; i++) mm(sum, sum, sum);
  memcpy(out, sum, sizeof sum);
}

/* H = sum_a w[a] lambda_a / 2 (Gell-Mann matrices), Hermitian traceless */
static void gellmann_combo(const double *w, cplx *h) {
  const double r3 = 1.0 / sqrt(3.0);
  for (int i = 0; i < 9; i++) { h[i].re = 0; h[i].im = 0; }
  /* lambda_1: (0,1),(1,0) = 1 */
  h[1].re += w[0]; h[3].re += w[0];
  /* lambda_2: (0,1) = -i, (1,0) = +i */
  h[1].im += -w[1]; h[3].im += w[1];
  /* lambda_3: diag(1,-1,0) */
  h[0].re += w[2]; h[4].re -= w[2];
  /* lambda_4: (0,2),(2,0) = 1 */
  h[2].re += w[3]; h[6].re += w[3];
  /* lambda_5: (0,2) = -i, (2,0) = +i */
  h[2].im += -w[4]; h[6].im += w[4];
  /* lambda_6: (1,2),(2,1) = 1 */
  h[5].re += w[5]; h[7].re += w[5];
  /* lambda_7: (1,2) = -i, (2,1) = +i */
  h[5].im += -w[6]; h[7].im += w[6];
  /* lambda_8: diag(1,1,-2)/sqrt(3) */
  h[0].re += w[7] * r3; h[4].re += w[7] * r3; h[8].re -= 2 * w[7] * r3;
  for (int i = 0; i < 9; i++) { h[i].re *= 0.5; h[i].im *= 0.5; }
}

/* exp(i eps H) with H from 8 normal deviates of stream (seed, 8*idx + a) */
static void random_su3(uint64_t seed, uint64_t idx, double eps, cplx *u) {
  double w[8];
  cplx h[9], x[9];
  for (int a = 0; a < 8; a++) w[a] = gauss(seed, 8 * idx + (uint64_t)a);
  gellmann_combo(w, h);
  for (int i = 0; i < 9; i++) { x[i].re = -eps * h[i].im; x[i].im = eps * h[i].re; }
  expm3(x, u);
}

static inline long site_shift(const int *d, long n, int mu, int step) {
  /* d = {T, Z, Y, X}; mu 0:x 1:y 2:z 3:t */
  long x = n % d[3], r = n / d[3];
  long y = r % d[2]; r /= d[2];
  long z = r % d[1];
  long t = r / d[1];
  long c[4] = {x, y, z, t};
  long L[4] = {d[3], d[2], d[1], d[0]};
  c[mu] = (c[mu] + step + L[mu]) % L[mu];
  return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
}

static void stout_step(const int *d, long V, double rho, const cplx *U, cplx *Unew) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < V; n++) {
    for (int mu = 0; mu < 4; mu++) {
      cplx C[9], t1[9], t2[9];
      for (int i = 0; i < 9; i++) { C[i].re = 0; C[i].im = 0; }
      long npm = site_shift(d, n, mu, +1);
      for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        long npn = site_shift(d, n, nu, +1);
        long nmn = site_shift(d, n, nu, -1);
        long nmn_pm = site_shift(d, nmn, mu, +1);
        /* upper staple U_nu(n) U_mu(n+nu) U_nu(n+mu)^dagger */
        mm(U + (n * 4 + nu) * 9, U + (npn * 4 + mu) * 9, t1);
        mmd(t1, U + (npm * 4 + nu) * 9, t2);
        for (int i = 0; i < 9; i++) { C[i].re += t2[i].re; C[i].im += t2[i].im; }
        /* lower staple U_nu(n-nu)^dagger U_mu(n-nu) U_nu(n-nu+mu) */
        mdm(U + (nmn * 4 + nu) * 9, U + (nmn * 4 + mu) * 9, t1);
        mm(t1, U + (nmn_pm * 4 + nu) * 9, t2);
        for (int i = 0; i < 9; i++) { C[i].re += t2[i].re; C[i].im += t2[i].im; }
      }
      for (int i = 0; i < 9; i++) { C[i].re *= rho; C[i].im *= rho; }
      const cplx *u = U + (n * 4 + mu) * 9;
      cplx Om[9], Omd[9], A[9], Q[9], iQ[9], E[9];
      mmd(C, u, Om);               /* Omega = C U^dagger */
      dag(Om, Omd);
      for (int i = 0; i < 9; i++) { A[i].re = Omd[i].re - Om[i].re; A[i].im = Omd[i].im - Om[i].im; }
      cplx tr = {A[0].re + A[4].re + A[8].re, A[0].im + A[4].im + A[8].im};
      /* Q = (i/2) A - (i/6) tr(A) 1 */
      for (int i = 0; i < 9; i++) {
        cplx v = A[i];
        if (i % 4 == 0) { v.re -= tr.re / 3.0; v.im -= tr.im / 3.0; }
        Q[i].re = -0.5 * v.im; Q[i].im = 0.5 * v.re;
      }
      for (int i = 0; i < 9; i++) { iQ[i].re = -Q[i].im; iQ[i].im = Q[i].re; }
      expm3(iQ, E);
      mm(E, u, Unew + (n * 4 + mu) * 9);
    }
  }
}

/* Public entry points. Return 0 on success, -1 on bad arguments or no memory. */

int synth_gauge(const int dims[4], double eps, int n_stout, double rho, uint64_t seed, double *links) {
  if (!dims || !links || n_stout < 0) return -1;
  long V = 1;
  for (int i = 0; i < 4; i++) { if (dims[i] < 1) return -1; V *= dims[i]; }
  cplx *U = (cplx *)links;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < V; n++)
    for (int mu = 0; mu < 4; mu++) random_su3(seed, (uint64_t)(n * 4 + mu), eps, U + (n * 4 + mu) * 9);
  if (n_stout == 0) return 0;
  cplx *tmp = (cplx *)malloc(sizeof(cplx) * 36 * (size_t)V);
  if (!tmp) return -1;
  for (int s = 0; s < n_stout; s++) {
    stout_step(dims, V, rho, U, tmp);
    memcpy(U, tmp, sizeof(cplx) * 36 * (size_t)V);
  }
  free(tmp);
  return 0;
}

/* One random SU(3) matrix exp(i eps H) per site: a gauge transformation G(n). */
int synth_su3_field(long V, double eps, uint64_t seed, double *g) {
  if (V < 0 || !g) return -1;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < V; n++) random_su3(seed, (uint64_t)n, eps, (cplx *)g + n * 9);
  return 0;
}

/* n independent N(0,1) reals (a complex vector of n/2 entries). */
int synth_gaussian(long n, uint64_t seed, double *out) {
  if (n < 0 || !out) return -1;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) out[i] = gauss(seed, (uint64_t)i);
  return 0;
}

/* n complex Z2 noise entries (+-1 +- i)/sqrt(2). */
int synth_z2(long n, uint64_t seed, double *out) {
  if (n < 0 || !out) return -1;
  const double s = 0.70710678118654752440084436210485;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; i++) {
    uint64_t v = sm64(seed * 0x9E3779B97F4A7C15ULL + (uint64_t)i);
    out[2 * i] = (v & 1) ? s : -s;
    out[2 * i + 1] = (v & 2) ? s : -s;
  }
  return 0;
}

/* n uniform deviates in (0, 1]. */
int synth_uniform(long n, uint64_t seed, double *out) {
  if (n < 0 || !out) return -1;
  for (long i = 0; i < n; i++) out[i] = unif(seed, (uint64_t)i);
  return 0;
}
