/*
 * FP64 CPU oracle for the Wilson-clover SAP-FGMRES hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark may load this library. It shares no code, header,
 * table or constant with the GPU path; the GPU library never calls it.
 *
 * Everything here is written for checking by eye, not for speed: full 4x4
 * gamma matrices, full 12x12 site matrices, plain loops in double precision.
 *
 * The paper (arXiv:1710.07041) names the method but defines none of its
 * formulas: Sec. 1 cites DD-alpha-AMG for "the discretized form of the Dirac
 * equation", Sec. 3.1 names "the MR inversion within a domain" (Table 1) and
 * "the entire Schwarz method" (Table 2) as the two important code parts. The
 * definitions below are the textbook ones that DD-alpha-AMG uses:
 *
 *  Wilson-clover operator (Sheikholeslami-Wohlert):
 *    (D psi)(n) = A(n) psi(n)
 *      - 1/2 sum_mu [ (1 - g_mu) U_mu(n) psi(n+mu) + (1 + g_mu) U_mu(n-mu)^+ psi(n-mu) ]
 *    A(n) = (4 + m0) + C(n)
 *    C(n) = -(c_sw/32) sum_{mu,nu} (g_mu g_nu) (x) (Q_mu,nu(n) - Q_nu,mu(n))
 *    Q_mu,nu(n) = sum of the four plaquette leaves at n in the (mu,nu) plane,
 *    all traversed mu-then-nu (counter-clockwise).
 *    Hops that cross the time boundary get a factor -1 (antiperiodic time);
 *    the clover leaves never carry that factor.
 *  Gamma matrices, chiral basis:  g_k = [[0, -i s_k], [i s_k, 0]] (k = x,y,z),
 *    g_t = [[0, 1], [1, 0]], with s_k the Pauli matrices. Then
 *    g5 = g_x g_y g_z g_t = diag(1, 1, -1, -1).
 *  Schwarz alternating procedure (multiplicative, red-black): blocks coloured
 *    by the parity of their block coordinates; per sweep, colour 0 then 1:
 *    r = b - D x, then for every block B of that colour x_B += D_B^-1 r_B
 *    (approximately), where D_B is D restricted to B with every hop that leaves
 *    B dropped.
 *  Block solve: even-odd Schur complement on odd sites,
 *    Dhat = A_oo - D_oe A_ee^-1 D_eo,  bhat = r_o - D_oe A_ee^-1 r_e,
 *    n_MR minimal-residual steps from e_o = 0:
 *      p = Dhat rho, alpha = <p,rho>/<p,p>, e_o += alpha rho, rho -= alpha p,
 *    then e_e = A_ee^-1 (r_e - D_eo e_o).
 *  FGMRES(m) (Saad 1993), right-preconditioned by the Schwarz method, modified
 *    Gram-Schmidt and complex Givens rotations; the true residual b - D x is
 *    recomputed at the end of each cycle and decides convergence.
 *
 * Layouts (complex double = [re, im]):
 *   dims {T, Z, Y, X}; site n = x + X*(y + Y*(z + Z*t)); mu = 0:x 1:y 2:z 3:t
 *   links   [V][4][3][3]     spinor [V][4][3]     site matrix [V][12][12]
 *   spin-colour index a = 3*spin + colour.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cd;

typedef struct {
  int L[4];   /* extents by direction: L[0]=X, L[1]=Y, L[2]=Z, L[3]=T */
  long V;
  int antiperiodic;
} lat_t;

static int lat_init(lat_t *lt, const int dims[4], int antiperiodic) {
  if (!dims) return -1;
  lt->L[0] = dims[3]; lt->L[1] = dims[2]; lt->L[2] = dims[1]; lt->L[3] = dims[0];
  lt->V = 1;
  for (int i = 0; i < 4; i++) {
    if (lt->L[i] < 1) return -1;
    lt->V *= lt->L[i];
  }
  lt->antiperiodic = antiperiodic;
  return 0;
}

static void coords(const lat_t *lt, long n, int c[4]) {
  for (int mu = 0; mu < 4; mu++) { c[mu] = (int)(n % lt->L[mu]); n /= lt->L[mu]; }
}
static long index_of(const lat_t *lt, const int c[4]) {
  return c[0] + (long)lt->L[0] * (c[1] + (long)lt->L[1] * (c[2] + (long)lt->L[2] * c[3]));
}
/* neighbour n +- mu; *sign = -1 when the hop crosses the antiperiodic time edge */
static long neighbour(const lat_t *lt, long n, int mu, int dir, double *sign) {
  int c[4];
  coords(lt, n, c);
  int v = c[mu] + dir;
  *sign = 1.0;
  if (v < 0 || v >= lt->L[mu]) {
    v = (v + lt->L[mu]) % lt->L[mu];
    if (mu == 3 && lt->antiperiodic) *sign = -1.0;
  }
  c[mu] = v;
  return index_of(lt, c);
}

/* ---------------------------------------------------------------- gammas */
static void pauli(int k, cd s[2][2]) {
  s[0][0] = s[0][1] = s[1][0] = s[1][1] = 0;
  if (k == 1) { s[0][1] = 1; s[1][0] = 1; }
  if (k == 2) { s[0][1] = -I; s[1][0] = I; }
  if (k == 3) { s[0][0] = 1; s[1][1] = -1; }
}

static void gamma_mu(int mu, cd g[4][4]) {
  memset(g, 0, sizeof(cd) * 16);
  if (mu == 3) {
    for (int i = 0; i < 2; i++) { g[i][2 + i] = 1; g[2 + i][i] = 1; }
    return;
  }
  cd s[2][2];
  pauli(mu + 1, s);
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      g[i][2 + j] = -I * s[i][j];
      g[2 + i][j] = I * s[i][j];
    }
}

static void mat4_mul(cd a[4][4], cd b[4][4], cd o[4][4]) {
  cd t[4][4];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      cd s = 0;
      for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
      t[i][j] = s;
    }
  memcpy(o, t, sizeof t);
}

/* mu = 0..3: gamma_mu; mu = 4: gamma5 = g_x g_y g_z g_t (computed) */
int or_gamma(int mu, double *out) {
  cd g[4][4];
  if (mu < 0 || mu > 4) return -1;
  if (mu < 4) {
    gamma_mu(mu, g);
  } else {
    cd t[4][4];
    gamma_mu(0, g);
    for (int k = 1; k < 4; k++) { gamma_mu(k, t); mat4_mul(g, t, g); }
  }
  memcpy(out, g, sizeof g);
  return 0;
}

/* ----------------------------------------------------------- colour algebra */
typedef struct { cd m[3][3]; } su3;

static su3 ld(const double *U, long n, int mu) {
  su3 r;
  memcpy(r.m, U + (n * 4 + mu) * 18, sizeof r.m);
  return r;
}
static su3 mul(su3 a, su3 b) {
  su3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cd s = 0;
      for (int k = 0; k < 3; k++) s += a.m[i][k] * b.m[k][j];
      r.m[i][j] = s;
    }
  return r;
}
static su3 dagger(su3 a) {
  su3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r.m[i][j] = conj(a.m[j][i]);
  return r;
}

/* --------------------------------------------------------------- clover */
static su3 shifted_link(const lat_t *lt, const double *U, long n, int a, int da, int b, int db, int mu) {
  double s;
  long m = n;
  if (da) m = neighbour(lt, m, a, da, &s);
  if (db) m = neighbour(lt, m, b, db, &s);
  return ld(U, m, mu);
}

/* sum of the four leaves at n in the (mu,nu) plane, each traversed mu then nu */
static su3 clover_leaves(const lat_t *lt, const double *U, long n, int mu, int nu) {
  su3 q, l;
  /* leaf 1: n -> n+mu -> n+mu+nu -> n+nu -> n */
  l = mul(mul(mul(ld(U, n, mu), shifted_link(lt, U, n, mu, 1, nu, 0, nu)),
              dagger(shifted_link(lt, U, n, nu, 1, mu, 0, mu))),
          dagger(ld(U, n, nu)));
  q = l;
  /* leaf 2: n -> n+nu -> n+nu-mu -> n-mu -> n */
  l = mul(mul(mul(ld(U, n, nu), dagger(shifted_link(lt, U, n, nu, 1, mu, -1, mu))),
              dagger(shifted_link(lt, U, n, mu, -1, nu, 0, nu))),
          shifted_link(lt, U, n, mu, -1, nu, 0, mu));
  for (int i = 0; i < 9; i++) q.m[i / 3][i % 3] += l.m[i / 3][i % 3];
  /* leaf 3: n -> n-mu -> n-mu-nu -> n-nu -> n */
  l = mul(mul(mul(dagger(shifted_link(lt, U, n, mu, -1, nu, 0, mu)),
                  dagger(shifted_link(lt, U, n, mu, -1, nu, -1, nu))),
              shifted_link(lt, U, n, mu, -1, nu, -1, mu)),
          shifted_link(lt, U, n, nu, -1, mu, 0, nu));
  for (int i = 0; i < 9; i++) q.m[i / 3][i % 3] += l.m[i / 3][i % 3];
  /* leaf 4: n -> n-nu -> n-nu+mu -> n+mu -> n */
  l = mul(mul(mul(dagger(shifted_link(lt, U, n, nu, -1, mu, 0, nu)),
                  shifted_link(lt, U, n, nu, -1, mu, 0, mu)),
              shifted_link(lt, U, n, nu, -1, mu, 1, nu)),
          dagger(ld(U, n, mu)));
  for (int i = 0; i < 9; i++) q.m[i / 3][i % 3] += l.m[i / 3][i % 3];
  return q;
}

/* C(n) as a 12x12 matrix per site, index 3*spin + colour */
int or_clover_term(const int dims[4], const double *U, double c_sw, double *Cout) {
  lat_t lt;
  if (lat_init(&lt, dims, 0) || !U || !Cout) return -1;
  cd gm[4][4][4];
  for (int mu = 0; mu < 4; mu++) gamma_mu(mu, gm[mu]);
#pragma omp parallel for schedule(static)
  for (long n = 0; n < lt.V; n++) {
    cd *C = (cd *)Cout + n * 144;
    for (int i = 0; i < 144; i++) C[i] = 0;
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) {
        if (mu == nu) continue;
        su3 qmn = clover_leaves(&lt, U, n, mu, nu);
        su3 qnm = clover_leaves(&lt, U, n, nu, mu);
        cd gg[4][4];
        mat4_mul(gm[mu], gm[nu], gg);
        for (int s = 0; s < 4; s++)
          for (int t = 0; t < 4; t++)
            for (int a = 0; a < 3; a++)
              for (int b = 0; b < 3; b++)
                C[(3 * s + a) * 12 + 3 * t + b] +=
                    -(c_sw / 32.0) * gg[s][t] * (qmn.m[a][b] - qnm.m[a][b]);
      }
  }
  return 0;
}

/* A(n) = (4 + m0) 1 + C(n) */
int or_site_matrix(long V, const double *C, double m0, double *A) {
  if (V < 0 || !C || !A) return -1;
  for (long n = 0; n < V; n++) {
    const cd *c = (const cd *)C + n * 144;
    cd *a = (cd *)A + n * 144;
    for (int i = 0; i < 144; i++) a[i] = c[i] + ((i % 13 == 0) ? (4.0 + m0) : 0.0);
  }
  return 0;
}

/* Gauss-Jordan inverse of one 12x12 complex matrix, partial pivoting */
static int inv12(const cd *m, cd *out) {
  cd a[12][24];
  for (int i = 0; i < 12; i++)
    for (int j = 0; j < 24; j++) a[i][j] = (j < 12) ? m[i * 12 + j] : (j - 12 == i ? 1.0 : 0.0);
  for (int c = 0; c < 12; c++) {
    int p = c;
    for (int r = c + 1; r < 12; r++)
      if (cabs(a[r][c]) > cabs(a[p][c])) p = r;
    if (cabs(a[p][c]) == 0) return -1;
    if (p != c)
      for (int j = 0; j < 24; j++) { cd t = a[c][j]; a[c][j] = a[p][j]; a[p][j] = t; }
    cd piv = a[c][c];
    for (int j = 0; j < 24; j++) a[c][j] /= piv;
    for (int r = 0; r < 12; r++) {
      if (r == c) continue;
      cd f = a[r][c];
      if (f != 0)
        for (int j = 0; j < 24; j++) a[r][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < 12; i++)
    for (int j = 0; j < 12; j++) out[i * 12 + j] = a[i][12 + j];
  return 0;
}

int or_site_inverse(long V, const double *A, double *Ainv) {
  if (V < 0 || !A || !Ainv) return -1;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long n = 0; n < V; n++) bad |= inv12((const cd *)A + n * 144, (cd *)Ainv + n * 144) != 0;
  return bad ? -2 : 0;
}

/* ----------------------------------------------------------- the operator */
/* out = M psi for one 12x12 site matrix */
static void site_mv(const cd *M, const cd *psi, cd *out) {
  for (int i = 0; i < 12; i++) {
    cd s = 0;
    for (int j = 0; j < 12; j++) s += M[i * 12 + j] * psi[j];
    out[i] = s;
  }
}

/* acc += -1/2 * sign * (1 -+ g_mu) (x) W psi, W = U or U^dagger */
static void hop_term(cd g[4][4], double pm, su3 W, double sign, const cd *psi, cd *acc) {
  cd up[4][3];
  for (int s = 0; s < 4; s++)
    for (int a = 0; a < 3; a++) {
      cd v = 0;
      for (int b = 0; b < 3; b++) v += W.m[a][b] * psi[3 * s + b];
      up[s][a] = v;
    }
  for (int s = 0; s < 4; s++)
    for (int a = 0; a < 3; a++) {
      cd v = up[s][a];
      for (int t = 0; t < 4; t++) v += pm * g[s][t] * up[t][a];
      acc[3 * s + a] += -0.5 * sign * v;
    }
}

/* hopping part at site n, counting only neighbours m with keep(m) */
typedef struct {
  const lat_t *lt;
  const int *bd;   /* block extents by direction, or NULL */
} nbr_filter;

static int same_block(const nbr_filter *f, long n, long m) {
  if (!f->bd) return 1;
  int cn[4], cm[4];
  coords(f->lt, n, cn);
  coords(f->lt, m, cm);
  for (int mu = 0; mu < 4; mu++)
    if (cn[mu] / f->bd[mu] != cm[mu] / f->bd[mu]) return 0;
  return 1;
}

static void hopping_at(const nbr_filter *f, const double *U, const cd *in, long n, cd *acc) {
  const lat_t *lt = f->lt;
  for (int mu = 0; mu < 4; mu++) {
    cd g[4][4];
    gamma_mu(mu, g);
    double sf, sb;
    long nf = neighbour(lt, n, mu, +1, &sf);
    long nb = neighbour(lt, n, mu, -1, &sb);
    if (same_block(f, n, nf)) hop_term(g, -1.0, ld(U, n, mu), sf, in + nf * 12, acc);
    if (same_block(f, n, nb)) hop_term(g, +1.0, dagger(ld(U, nb, mu)), sb, in + nb * 12, acc);
  }
}

int or_apply_D(const int dims[4], int antiperiodic, const double *U, const double *A,
               const double *in, double *out) {
  lat_t lt;
  if (lat_init(&lt, dims, antiperiodic) || !U || !A || !in || !out || in == out) return -1;
  nbr_filter f = {&lt, NULL};
#pragma omp parallel for schedule(static)
  for (long n = 0; n < lt.V; n++) {
    cd acc[12];
    site_mv((const cd *)A + n * 144, (const cd *)in + n * 12, acc);
    hopping_at(&f, U, (const cd *)in, n, acc);
    memcpy((cd *)out + n * 12, acc, sizeof acc);
  }
  return 0;
}

/* (D psi)(n) at the listed sites only, with A(n) = 4 + m0 + C(n) formed from
 * the links on the fly (same definitions as or_clover_term and or_apply_D).
 * For checking results on lattices whose full site matrices would not fit in
 * host memory. out: [nsites][12] complex. */
int or_apply_D_sites(const int dims[4], int antiperiodic, const double *U, double c_sw, double m0,
                     const double *in, const long *sites, long nsites, double *out) {
  lat_t lt;
  if (lat_init(&lt, dims, antiperiodic) || !U || !in || !sites || !out || nsites < 0) return -1;
  cd gm[4][4][4];
  for (int mu = 0; mu < 4; mu++) gamma_mu(mu, gm[mu]);
  nbr_filter f = {&lt, NULL};
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long i = 0; i < nsites; i++) {
    long n = sites[i];
    if (n < 0 || n >= lt.V) { bad = 1; continue; }
    cd A[144];
    for (int k = 0; k < 144; k++) A[k] = (k % 13 == 0) ? (4.0 + m0) : 0.0;
    for (int mu = 0; mu < 4; mu++)
      for (int nu = 0; nu < 4; nu++) {
        if (mu == nu) continue;
        su3 qmn = clover_leaves(&lt, U, n, mu, nu);
        su3 qnm = clover_leaves(&lt, U, n, nu, mu);
        cd gg[4][4];
        mat4_mul(gm[mu], gm[nu], gg);
        for (int s = 0; s < 4; s++)
          for (int t = 0; t < 4; t++)
            for (int a = 0; a < 3; a++)
              for (int b = 0; b < 3; b++)
                A[(3 * s + a) * 12 + 3 * t + b] += -(c_sw / 32.0) * gg[s][t] * (qmn.m[a][b] - qnm.m[a][b]);
      }
    cd acc[12];
    site_mv(A, (const cd *)in + n * 12, acc);
    hopping_at(&f, U, (const cd *)in, n, acc);
    memcpy((cd *)out + i * 12, acc, sizeof acc);
  }
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------- blocks */
typedef struct {
  lat_t lt;
  int bd[4];     /* block extents by direction (x, y, z, t) */
  int nb[4];     /* number of blocks by direction */
  long nblocks, vb;
} blocking_t;

static int blocking_init(blocking_t *B, const int dims[4], int antiperiodic, const int bdims[4]) {
  if (lat_init(&B->lt, dims, antiperiodic) || !bdims) return -1;
  B->nblocks = 1;
  B->vb = 1;
  for (int mu = 0; mu < 4; mu++) {
    B->bd[mu] = bdims[3 - mu];
    if (B->bd[mu] < 1 || B->lt.L[mu] % B->bd[mu]) return -1;
    B->nb[mu] = B->lt.L[mu] / B->bd[mu];
    B->nblocks *= B->nb[mu];
    B->vb *= B->bd[mu];
  }
  return 0;
}

/* site k (lexicographic inside the block, x fastest) of block b */
static long block_site(const blocking_t *B, long b, long k) {
  int bc[4], c[4];
  for (int mu = 0; mu < 4; mu++) { bc[mu] = (int)(b % B->nb[mu]); b /= B->nb[mu]; }
  for (int mu = 0; mu < 4; mu++) { c[mu] = bc[mu] * B->bd[mu] + (int)(k % B->bd[mu]); k /= B->bd[mu]; }
  return index_of(&B->lt, c);
}
static int block_colour(const blocking_t *B, long b) {
  int s = 0;
  for (int mu = 0; mu < 4; mu++) { s += (int)(b % B->nb[mu]); b /= B->nb[mu]; }
  return s & 1;
}
static int parity(const lat_t *lt, long n) {
  int c[4];
  coords(lt, n, c);
  return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* D_B restricted to block b: out_B = A psi_B + hops between sites of B only */
int or_apply_DB(const int dims[4], int antiperiodic, const int bdims[4], long block,
                const double *U, const double *A, const double *in, double *out) {
  blocking_t B;
  if (blocking_init(&B, dims, antiperiodic, bdims) || block < 0 || block >= B.nblocks) return -1;
  nbr_filter f = {&B.lt, B.bd};
  for (long k = 0; k < B.vb; k++) {
    long n = block_site(&B, block, k);
    cd acc[12];
    site_mv((const cd *)A + n * 144, (const cd *)in + n * 12, acc);
    hopping_at(&f, U, (const cd *)in, n, acc);
    memcpy((cd *)out + n * 12, acc, sizeof acc);
  }
  return 0;
}

/* local index (lexicographic inside its block) of global site n */
static long local_index(const blocking_t *B, long n) {
  int c[4];
  coords(&B->lt, n, c);
  long k = 0;
  for (int mu = 3; mu >= 0; mu--) k = k * B->bd[mu] + c[mu] % B->bd[mu];
  return k;
}

/* Block-local vectors are [vb][12], indexed by the local site k.
 * out[k] = hops between sites of block b, at the local sites k of parity p. */
static void block_hop(const blocking_t *B, long b, int p, const double *U, const cd *in, cd *out) {
  for (long k = 0; k < B->vb; k++) {
    long n = block_site(B, b, k);
    if (parity(&B->lt, n) != p) continue;
    cd acc[12] = {0};
    for (int mu = 0; mu < 4; mu++) {
      cd g[4][4];
      gamma_mu(mu, g);
      double sf, sb;
      long nf = neighbour(&B->lt, n, mu, +1, &sf);
      long nb = neighbour(&B->lt, n, mu, -1, &sb);
      nbr_filter f = {&B->lt, B->bd};
      if (same_block(&f, n, nf)) hop_term(g, -1.0, ld(U, n, mu), sf, in + local_index(B, nf) * 12, acc);
      if (same_block(&f, n, nb)) hop_term(g, +1.0, dagger(ld(U, nb, mu)), sb, in + local_index(B, nb) * 12, acc);
    }
    memcpy(out + k * 12, acc, sizeof acc);
  }
}
static void block_site_mv(const blocking_t *B, long b, int p, const double *M, const cd *in, cd *out) {
  for (long k = 0; k < B->vb; k++) {
    long n = block_site(B, b, k);
    if (parity(&B->lt, n) != p) continue;
    site_mv((const cd *)M + n * 144, in + k * 12, out + k * 12);
  }
}
static cd block_dot(const blocking_t *B, long b, int p, const cd *x, const cd *y) {
  cd s = 0;
  for (long k = 0; k < B->vb; k++) {
    if (parity(&B->lt, block_site(B, b, k)) != p) continue;
    for (int i = 0; i < 12; i++) s += conj(x[k * 12 + i]) * y[k * 12 + i];
  }
  return s;
}

/* Even-odd block solve with nmr MR steps on the odd-site Schur complement.
 * r, e: block-local right-hand side and result; w: five block-local scratch
 * vectors [5][vb][12]. */
static void block_mr(const blocking_t *B, long b, const double *U, const double *A, const double *Ainv,
                     const cd *r, cd *e, int nmr, cd *w) {
  long vb = B->vb;
  cd *t_e = w, *rho = w + 12 * vb, *p = w + 24 * vb, *q = w + 36 * vb, *s = w + 48 * vb;
  memset(w, 0, sizeof(cd) * 60 * vb);
  memset(e, 0, sizeof(cd) * 12 * vb);
  /* bhat_o = r_o - D_oe A_ee^-1 r_e */
  block_site_mv(B, b, 0, Ainv, r, t_e);
  block_hop(B, b, 1, U, t_e, q);
  for (long k = 0; k < vb; k++) {
    if (parity(&B->lt, block_site(B, b, k)) != 1) continue;
    for (int i = 0; i < 12; i++) rho[k * 12 + i] = r[k * 12 + i] - q[k * 12 + i];
  }
  for (int it = 0; it < nmr; it++) {
    /* p = Dhat rho = A_oo rho - D_oe A_ee^-1 D_eo rho */
    block_hop(B, b, 0, U, rho, q);
    block_site_mv(B, b, 0, Ainv, q, s);
    block_hop(B, b, 1, U, s, q);
    block_site_mv(B, b, 1, A, rho, p);
    for (long k = 0; k < vb; k++) {
      if (parity(&B->lt, block_site(B, b, k)) != 1) continue;
      for (int i = 0; i < 12; i++) p[k * 12 + i] -= q[k * 12 + i];
    }
    cd pr = block_dot(B, b, 1, p, rho);
    double pp = creal(block_dot(B, b, 1, p, p));
    if (pp == 0) break;
    cd alpha = pr / pp;
    for (long k = 0; k < vb; k++) {
      if (parity(&B->lt, block_site(B, b, k)) != 1) continue;
      for (int i = 0; i < 12; i++) {
        e[k * 12 + i] += alpha * rho[k * 12 + i];
        rho[k * 12 + i] -= alpha * p[k * 12 + i];
      }
    }
  }
  /* e_e = A_ee^-1 (r_e - D_eo e_o) */
  block_hop(B, b, 0, U, e, q);
  for (long k = 0; k < vb; k++) {
    if (parity(&B->lt, block_site(B, b, k)) != 0) continue;
    for (int i = 0; i < 12; i++) s[k * 12 + i] = r[k * 12 + i] - q[k * 12 + i];
  }
  block_site_mv(B, b, 0, Ainv, s, t_e);
  for (long k = 0; k < vb; k++) {
    if (parity(&B->lt, block_site(B, b, k)) != 0) continue;
    for (int i = 0; i < 12; i++) e[k * 12 + i] = t_e[k * 12 + i];
  }
}

/* Block solve of one block (for tests): e_B ~= D_B^-1 r_B with nmr MR steps.
 * r and e are full-lattice vectors; only the block's sites are read/written. */
int or_block_solve(const int dims[4], int antiperiodic, const int bdims[4], long block,
                   const double *U, const double *A, const double *Ainv,
                   const double *r, double *e, int nmr) {
  blocking_t B;
  if (blocking_init(&B, dims, antiperiodic, bdims) || block < 0 || block >= B.nblocks) return -1;
  cd *w = (cd *)calloc((size_t)B.vb * 84, sizeof(cd));
  if (!w) return -2;
  cd *rl = w + 60 * B.vb, *el = w + 72 * B.vb;
  for (long k = 0; k < B.vb; k++)
    memcpy(rl + k * 12, (const cd *)r + block_site(&B, block, k) * 12, sizeof(cd) * 12);
  block_mr(&B, block, U, A, Ainv, rl, el, nmr, w);
  for (long k = 0; k < B.vb; k++)
    memcpy((cd *)e + block_site(&B, block, k) * 12, el + k * 12, sizeof(cd) * 12);
  free(w);
  return 0;
}

int or_block_colour(const int dims[4], const int bdims[4], long block) {
  blocking_t B;
  if (blocking_init(&B, dims, 0, bdims) || block < 0 || block >= B.nblocks) return -1;
  return block_colour(&B, block);
}

long or_block_site(const int dims[4], const int bdims[4], long block, long k) {
  blocking_t B;
  if (blocking_init(&B, dims, 0, bdims) || block < 0 || block >= B.nblocks || k < 0 || k >= B.vb) return -1;
  return block_site(&B, block, k);
}

/* Schwarz sweeps: x is updated in place (x = 0 on entry gives the preconditioner). */
static int sap_run(const blocking_t *B, const double *U, const double *A, const double *Ainv,
                   const cd *b, cd *x, int nsweep, int nmr) {
  long V = B->lt.V;
  for (int mu = 0; mu < 4; mu++)
    if (B->nb[mu] % 2) return -1;   /* red-black colouring needs even block counts */
  int dims[4] = {B->lt.L[3], B->lt.L[2], B->lt.L[1], B->lt.L[0]};
  cd *r = (cd *)malloc(sizeof(cd) * 12 * V);
  if (!r) return -2;
  int bad = 0;
  for (int sw = 0; sw < nsweep; sw++)
    for (int colour = 0; colour < 2; colour++) {
      /* r = b - D x with the current x */
      or_apply_D(dims, B->lt.antiperiodic, U, A, (const double *)x, (double *)r);
      for (long i = 0; i < 12 * V; i++) r[i] = b[i] - r[i];
#pragma omp parallel reduction(| : bad)
      {
        cd *w = (cd *)malloc(sizeof(cd) * 84 * B->vb);
        if (!w) bad = 1;
#pragma omp for schedule(dynamic)
        for (long blk = 0; blk < B->nblocks; blk++) {
          if (!w || block_colour(B, blk) != colour) continue;
          cd *rl = w + 60 * B->vb, *el = w + 72 * B->vb;
          for (long k = 0; k < B->vb; k++)
            memcpy(rl + k * 12, r + block_site(B, blk, k) * 12, sizeof(cd) * 12);
          block_mr(B, blk, U, A, Ainv, rl, el, nmr, w);
          for (long k = 0; k < B->vb; k++) {
            long n = block_site(B, blk, k);
            for (int i = 0; i < 12; i++) x[n * 12 + i] += el[k * 12 + i];
          }
        }
        free(w);
      }
    }
  free(r);
  return bad ? -2 : 0;
}

int or_sap(const int dims[4], int antiperiodic, const int bdims[4], const double *U, const double *A,
           const double *Ainv, const double *b, double *x, int nsweep, int nmr) {
  blocking_t B;
  if (blocking_init(&B, dims, antiperiodic, bdims) || !U || !A || !Ainv || !b || !x) return -1;
  return sap_run(&B, U, A, Ainv, (const cd *)b, (cd *)x, nsweep, nmr);
}

/* ------------------------------------------------------------- FGMRES */
static cd vdot(long n, const cd *a, const cd *b) {
  cd s = 0;
  for (long i = 0; i < n; i++) s += conj(a[i]) * b[i];
  return s;
}
static double vnorm(long n, const cd *a) { return sqrt(creal(vdot(n, a, a))); }

/* Modified Gram-Schmidt step of the Arnoldi process: w is projected against
 * the basis vectors v_0 .. v_{k-1} (V holds them back to back, n complex
 * each) in order, h_i = <v_i, w> taken after the previous projections. */
static void mgs_project(long n, const cd *V, int k, cd *w, cd *h) {
  for (int i = 0; i < k; i++) {
    const cd *v = V + (long)i * n;
    h[i] = vdot(n, v, w);
    for (long l = 0; l < n; l++) w[l] -= h[i] * v[l];
  }
}

/* The same step on caller arrays (for timing and tests): w and h (k complex)
 * are overwritten. */
int or_gram_schmidt(long n, const double *V, int k, double *w, double *h) {
  if (n < 1 || k < 0 || !V || !w || (k > 0 && !h)) return -1;
  mgs_project(n, (const cd *)V, k, (cd *)w, (cd *)h);
  return 0;
}

/* OpenMP threads used by the parallel loops from now on (n >= 1; n <= 0
 * leaves the setting unchanged). Returns the number in effect. */
int omp_get_max_threads(void);
void omp_set_num_threads(int);
int or_set_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
}

/* FGMRES(m) right-preconditioned by SAP (nsweep sweeps, nmr MR steps, x0 = 0 per
 * application). x holds the initial guess on entry and the solution on exit.
 * stats[0] = preconditioner applications, stats[1] = restart cycles,
 * stats[2] = final true relative residual. Returns 0 when converged, 1 when
 * max_iter was reached, <0 on errors. */
int or_fgmres(const int dims[4], int antiperiodic, const int bdims[4], const double *U,
              const double *A, const double *Ainv, const double *bv, double *xv,
              int m, double tol, int max_iter, int nsweep, int nmr, double *stats) {
  blocking_t B;
  if (blocking_init(&B, dims, antiperiodic, bdims) || m < 1 || !bv || !xv) return -1;
  long n = 12 * B.lt.V;
  const cd *b = (const cd *)bv;
  cd *x = (cd *)xv;
  cd *Vb = (cd *)malloc(sizeof(cd) * n * (m + 1));
  cd *Z = (cd *)malloc(sizeof(cd) * n * m);
  cd *w = (cd *)malloc(sizeof(cd) * n);
  cd *H = (cd *)calloc((size_t)(m + 1) * m, sizeof(cd));
  cd *g = (cd *)calloc(m + 1, sizeof(cd));
  double *cs = (double *)calloc(m, sizeof(double));
  cd *sn = (cd *)calloc(m, sizeof(cd));
  cd *y = (cd *)calloc(m, sizeof(cd));
  int rc = 1, its = 0, cycles = 0;
  double bnorm = vnorm(n, b), rel = 1.0;
  if (!Vb || !Z || !w || !H || !g || !cs || !sn || !y) { rc = -2; goto done; }
  if (bnorm == 0) {
    memset(x, 0, sizeof(cd) * n);
    rel = 0; rc = 0;
    goto done;
  }
  int dd[4] = {dims[0], dims[1], dims[2], dims[3]};
  for (;;) {
    /* true residual */
    or_apply_D(dd, antiperiodic, U, A, (const double *)x, (double *)w);
    for (long i = 0; i < n; i++) w[i] = b[i] - w[i];
    double beta = vnorm(n, w);
    rel = beta / bnorm;
    if (rel <= tol) { rc = 0; break; }
    if (its >= max_iter) { rc = 1; break; }
    cycles++;
    for (long i = 0; i < n; i++) Vb[i] = w[i] / beta;
    memset(g, 0, sizeof(cd) * (m + 1));
    g[0] = beta;
    int j, k = 0;
    for (j = 0; j < m && its < max_iter; j++) {
      cd *v = Vb + (long)j * n, *z = Z + (long)j * n;
      memset(z, 0, sizeof(cd) * n);
      if (sap_run(&B, U, A, Ainv, v, z, nsweep, nmr)) { rc = -2; goto done; }
      its++;
      or_apply_D(dd, antiperiodic, U, A, (const double *)z, (double *)w);
      cd hcol[j + 1];
      mgs_project(n, Vb, j + 1, w, hcol);
      for (int i = 0; i <= j; i++) H[i * m + j] = hcol[i];
      double hn = vnorm(n, w);
      H[(j + 1) * m + j] = hn;
      if (hn > 0)
        for (long l = 0; l < n; l++) Vb[(long)(j + 1) * n + l] = w[l] / hn;
      /* previous rotations on column j */
      for (int i = 0; i < j; i++) {
        cd a = H[i * m + j], c2 = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c2;
        H[(i + 1) * m + j] = -conj(sn[i]) * a + cs[i] * c2;
      }
      /* new rotation zeroing H[j+1][j] */
      cd a = H[j * m + j];
      double bb = creal(H[(j + 1) * m + j]);
      double r = sqrt(creal(a * conj(a)) + bb * bb);
      if (cabs(a) == 0) { cs[j] = 0; sn[j] = 1; }
      else { cs[j] = cabs(a) / r; sn[j] = (a / cabs(a)) * bb / r; }
      H[j * m + j] = cs[j] * a + sn[j] * bb;
      H[(j + 1) * m + j] = 0;
      g[j + 1] = -conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (cabs(g[j + 1]) <= tol * bnorm || hn == 0) break;
    }
    /* back substitution R y = g, then x += Z y */
    for (int i = k - 1; i >= 0; i--) {
      cd s = g[i];
      for (int l = i + 1; l < k; l++) s -= H[i * m + l] * y[l];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < k; i++)
      for (long l = 0; l < n; l++) x[l] += y[i] * Z[(long)i * n + l];
  }
done:
  if (stats) { stats[0] = its; stats[1] = cycles; stats[2] = rel; }
  free(Vb); free(Z); free(w); free(H); free(g); free(cs); free(sn); free(y);
  return rc;
}
