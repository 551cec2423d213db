/*
 * oracle.c -- plain FP64 CPU oracle (test infrastructure; see oracle.h).
 *
 * Every routine is the textbook definition written out, in the order the paper
 * states it, with no blocking or reordering.  Compile with -ffp-contract=off so
 * that a*b+c is never fused: the oracle is a predictable FP64 reference.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ======================================================================== */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11, Sec. 3.2: ten rounds of two 32x32->64 products, */
/* the key bumped by the Weyl constants between rounds.                     */
/* ======================================================================== */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in the open interval (0,1): the top 52 bits x of the 64-bit word give
 * u = (x + 1/2) 2^-52, an odd multiple of 2^-53.  x + 1/2 needs 53 significant bits,
 * so it is exact in FP64, and u never rounds to 0 or 1. */
double orc_uniform53(uint32_t hi, uint32_t lo) {
  uint64_t x = (((uint64_t)hi << 32) | (uint64_t)lo) >> 12;
  return ((double)x + 0.5) * (1.0 / 4503599627370496.0);
}

static void philox_for(uint64_t seed, uint32_t sweep, uint32_t particle, uint32_t purpose,
                       uint32_t j, uint32_t out[4]) {
  uint32_t ctr[4] = {sweep, particle, purpose, j};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* Box-Muller: (u1, u2) -> sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2) */
void orc_normal3(uint64_t seed, uint32_t sweep, uint32_t particle, uint32_t purpose,
                 double z[3]) {
  uint32_t w[4];
  philox_for(seed, sweep, particle, purpose, 0u, w);
  double u1 = orc_uniform53(w[0], w[1]);
  double u2 = orc_uniform53(w[2], w[3]);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 2.0 * M_PI * u2;
  z[0] = rad * cos(ang);
  z[1] = rad * sin(ang);
  philox_for(seed, sweep, particle, purpose, 1u, w);
  u1 = orc_uniform53(w[0], w[1]);
  u2 = orc_uniform53(w[2], w[3]);
  rad = sqrt(-2.0 * log(u1));
  ang = 2.0 * M_PI * u2;
  z[2] = rad * cos(ang);
}

double orc_accept_uniform(uint64_t seed, uint32_t sweep, uint32_t particle) {
  uint32_t w[4];
  philox_for(seed, sweep, particle, 2u, 0u, w);
  return orc_uniform53(w[0], w[1]);
}

/* ======================================================================== */
/* Geometry: orbital centres on a periodic lattice (Sec. 2.1 and Sec. 4).    */
/* ======================================================================== */
int orc_n(const orc_system* s) {
  int c = s->K * s->K * s->K;
  return s->lattice == 1 ? 2 * c : c;
}

static double box_len(const orc_system* s) { return (double)s->K * s->a; }

void orc_sites(const orc_system* s, double* Z) {
  int K = s->K;
  int per = s->lattice == 1 ? 2 : 1;
  for (int jz = 0; jz < K; ++jz)
    for (int jy = 0; jy < K; ++jy)
      for (int jx = 0; jx < K; ++jx) {
        int cell = jx + K * (jy + K * jz);
        for (int b = 0; b < per; ++b) {
          int j = cell * per + b;
          double off = 0.5 * (double)b;
          Z[3 * j + 0] = s->a * ((double)jx + off);
          Z[3 * j + 1] = s->a * ((double)jy + off);
          Z[3 * j + 2] = s->a * ((double)jz + off);
        }
      }
}

/* wrap x into the periodic box [0, L) */
static double wrap(double x, double L) {
  double y = x - L * floor(x / L);
  if (y >= L) y -= L;
  return y;
}

/* minimum-image component */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

void orc_initial_positions(const orc_system* s, uint64_t seed, double jitter, double* R) {
  int n = orc_n(s);
  double L = box_len(s);
  double* Z = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  orc_sites(s, Z);
  for (int i = 0; i < n; ++i) {
    double z[3];
    orc_normal3(seed, 0u, (uint32_t)i, 0u, z);
    for (int d = 0; d < 3; ++d) R[3 * i + d] = wrap(Z[3 * i + d] + jitter * z[d], L);
  }
  free(Z);
}

void orc_propose(const orc_system* s, uint64_t seed, uint32_t sweep, uint32_t particle,
                 double sigma, const double r_old[3], double r_new[3]) {
  double z[3];
  double L = box_len(s);
  orc_normal3(seed, sweep, particle, 1u, z);
  for (int d = 0; d < 3; ++d) r_new[d] = wrap(r_old[d] + sigma * z[d], L);
}

/* phi_j(r) = exp(-kappa d^2) when d <= r_c (min image), else 0  (Eq. 3) */
static double orbital(const orc_system* s, const double* Zj, const double* r, double L,
                      double rc2) {
  double dx = min_image(r[0] - Zj[0], L);
  double dy = min_image(r[1] - Zj[1], L);
  double dz = min_image(r[2] - Zj[2], L);
  double d2 = dx * dx + dy * dy + dz * dz;
  if (d2 <= rc2) return exp(-s->kappa * d2);
  return 0.0;
}

void orc_row_dense(const orc_system* s, const double* Z, const double r[3], double* row) {
  int n = orc_n(s);
  double L = box_len(s);
  double rc2 = s->r_c * s->r_c;
  for (int j = 0; j < n; ++j) row[j] = orbital(s, Z + 3 * j, r, L, rc2);
}

void orc_slater_dense(const orc_system* s, const double* Z, const double* R, double* A) {
  int n = orc_n(s);
  for (int i = 0; i < n; ++i) orc_row_dense(s, Z, R + 3 * i, A + (size_t)i * n);
}

long orc_slater_csr(const orc_system* s, const double* Z, const double* R, long cap,
                    int64_t* rowptr, int32_t* col, double* val) {
  int n = orc_n(s);
  double L = box_len(s);
  double rc2 = s->r_c * s->r_c;
  long nnz = 0;
  rowptr[0] = 0;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double v = orbital(s, Z + 3 * j, R + 3 * i, L, rc2);
      if (v != 0.0) {
        if (nnz >= cap) return -1;
        col[nnz] = j;
        val[nnz] = v;
        ++nnz;
      }
    }
    rowptr[i + 1] = nnz;
  }
  return nnz;
}

/* ======================================================================== */
/* Dense linear algebra (Golub & Van Loan, Alg. 3.4.1: LU, partial pivoting) */
/* ======================================================================== */
int orc_lu(int n, double* A, int* piv, int* sign) {
  *sign = 1;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0) return 1;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
      *sign = -*sign;
    }
    double pivot = A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / pivot;
      A[(size_t)i * n + k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return 0;
}

void orc_lu_solve(int n, const double* LU, const int* piv, const double* b, double* x) {
  for (int i = 0; i < n; ++i) x[i] = b[i];
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int i = 0; i < n; ++i) {            /* L y = P b, unit lower */
    double acc = x[i];
    for (int j = 0; j < i; ++j) acc -= LU[(size_t)i * n + j] * x[j];
    x[i] = acc;
  }
  for (int i = n - 1; i >= 0; --i) {       /* U x = y */
    double acc = x[i];
    for (int j = i + 1; j < n; ++j) acc -= LU[(size_t)i * n + j] * x[j];
    x[i] = acc / LU[(size_t)i * n + i];
  }
}

double orc_lu_logabsdet(int n, const double* LU, int sign, int* det_sign) {
  double acc = 0.0;
  int sg = sign;
  for (int i = 0; i < n; ++i) {
    double d = LU[(size_t)i * n + i];
    if (d < 0.0) sg = -sg;
    acc += log(fabs(d));
  }
  *det_sign = sg;
  return acc;
}

/* Leibniz formula det A = sum_sigma sgn(sigma) prod_i a_{i,sigma(i)}; the
 * permutations are enumerated by Heap's algorithm, each step one transposition. */
double orc_leibniz_det(int n, const double* A) {
  if (n <= 0) return 1.0;
  int perm[16], c[16];
  for (int i = 0; i < n; ++i) { perm[i] = i; c[i] = 0; }
  int sgn = 1;
  double total = 0.0;
  for (;;) {
    double prod = (double)sgn;
    for (int i = 0; i < n; ++i) prod *= A[(size_t)i * n + perm[i]];
    total += prod;
    int i = 1;
    while (i < n && c[i] >= i) { c[i] = 0; ++i; }
    if (i >= n) break;
    int j = (i % 2 == 0) ? 0 : c[i];
    int t = perm[j]; perm[j] = perm[i]; perm[i] = t;
    sgn = -sgn;
    c[i] += 1;
  }
  return total;
}

int orc_ratio_dense(int n, const double* A, int i, const double* a_new, double* ratio,
                    double* ratio_logdet) {
  size_t nn = (size_t)n * n;
  double* LU = (double*)malloc(sizeof(double) * nn);
  int* piv = (int*)malloc(sizeof(int) * n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  double* z = (double*)malloc(sizeof(double) * n);
  int sign, rc = 0;
  memcpy(LU, A, sizeof(double) * nn);
  if (orc_lu(n, LU, piv, &sign)) { rc = 1; goto out; }
  e[i] = 1.0;
  orc_lu_solve(n, LU, piv, e, z);              /* A z = e_i */
  {
    double acc = 0.0;                          /* u^T z, u = a' - a_i */
    for (int j = 0; j < n; ++j) acc += (a_new[j] - A[(size_t)i * n + j]) * z[j];
    *ratio = 1.0 + acc;
  }
  if (ratio_logdet) {
    int s0, s1, sign1;
    double ld0 = orc_lu_logabsdet(n, LU, sign, &s0);
    memcpy(LU, A, sizeof(double) * nn);
    memcpy(LU + (size_t)i * n, a_new, sizeof(double) * n);
    if (orc_lu(n, LU, piv, &sign1)) {
      *ratio_logdet = 0.0;
    } else {
      double ld1 = orc_lu_logabsdet(n, LU, sign1, &s1);
      *ratio_logdet = (double)(s0 * s1) * exp(ld1 - ld0);
    }
  }
out:
  free(LU); free(piv); free(e); free(z);
  return rc;
}

int orc_inverse(int n, const double* A, double* B) {
  size_t nn = (size_t)n * n;
  double* LU = (double*)malloc(sizeof(double) * nn);
  int* piv = (int*)malloc(sizeof(int) * n);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  double* x = (double*)malloc(sizeof(double) * n);
  int sign, rc = 0;
  memcpy(LU, A, sizeof(double) * nn);
  if (orc_lu(n, LU, piv, &sign)) { rc = 1; goto out; }
  for (int j = 0; j < n; ++j) {
    e[j] = 1.0;
    orc_lu_solve(n, LU, piv, e, x);
    e[j] = 0.0;
    for (int i = 0; i < n; ++i) B[(size_t)i * n + j] = x[i];
  }
out:
  free(LU); free(piv); free(e); free(x);
  return rc;
}

/* standard algorithm (Sec. 1): ratio = 1 + u^T (A^{-1} e_i) = 1 + sum_j u_j B_ji */
double orc_sm_ratio(int n, const double* B, int i, const double* u) {
  double acc = 0.0;
  for (int j = 0; j < n; ++j) acc += u[j] * B[(size_t)j * n + i];
  return 1.0 + acc;
}

/* Sherman-Morrison for A' = A + e_i u^T:
 *   A'^{-1} = B - (B e_i)(u^T B) / (1 + u^T B e_i)                        */
void orc_sm_update(int n, double* B, int i, const double* u, double ratio, double* work) {
  double* colv = work;       /* B e_i   */
  double* rowv = work + n;   /* u^T B   */
  for (int a = 0; a < n; ++a) colv[a] = B[(size_t)a * n + i];
  for (int b = 0; b < n; ++b) rowv[b] = 0.0;
  for (int l = 0; l < n; ++l) {
    double ul = u[l];
    if (ul == 0.0) continue;
    for (int b = 0; b < n; ++b) rowv[b] += ul * B[(size_t)l * n + b];
  }
  for (int a = 0; a < n; ++a) {
    double f = colv[a] / ratio;
    if (f == 0.0) continue;
    for (int b = 0; b < n; ++b) B[(size_t)a * n + b] -= f * rowv[b];
  }
}

/* ======================================================================== */
/* Restarted GMRES (Saad & Schultz 1986), modified Gram-Schmidt, Givens      */
/* rotations, right Jacobi scaling x = D^{-1} y.  Plain reference solver.    */
/* ======================================================================== */
static void csr_mv(int n, const int64_t* rp, const int32_t* ci, const double* v,
                   const double* x, double* y) {
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) acc += v[t] * x[ci[t]];
    y[i] = acc;
  }
}

static double nrm2(int n, const double* x) {
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += x[i] * x[i];
  return sqrt(acc);
}

int orc_gmres(int n, const int64_t* rowptr, const int32_t* col, const double* val,
              const double* b, double* x, int restart, int max_iter, double tol) {
  int m = restart;
  double* dinv = (double*)malloc(sizeof(double) * n);
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * m);
  double* sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* y = (double*)malloc(sizeof(double) * m);
  double* w = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  int total = 0, result = -1;
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
      if (col[q] == i) d = val[q];
    dinv[i] = (d != 0.0) ? 1.0 / d : 1.0;
  }
  double bnorm = nrm2(n, b);
  if (bnorm == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    result = 0;
    goto out;
  }
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  while (total < max_iter) {
    csr_mv(n, rowptr, col, val, x, w);                       /* r = b - A x */
    for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
    double beta = nrm2(n, w);
    if (beta <= tol * bnorm) { result = total; break; }
    for (int i = 0; i < n; ++i) V[i] = w[i] / beta;
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta;
    int j = 0;
    for (; j < m && total < max_iter; ++j) {
      double* vj = V + (size_t)j * n;
      double* vn = V + (size_t)(j + 1) * n;
      for (int i = 0; i < n; ++i) t[i] = dinv[i] * vj[i];
      csr_mv(n, rowptr, col, val, t, vn);                    /* A D^{-1} v_j */
      for (int k = 0; k <= j; ++k) {                          /* MGS */
        double* vk = V + (size_t)k * n;
        double h = 0.0;
        for (int i = 0; i < n; ++i) h += vk[i] * vn[i];
        H[(size_t)k * m + j] = h;
        for (int i = 0; i < n; ++i) vn[i] -= h * vk[i];
      }
      double hn = nrm2(n, vn);
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (int i = 0; i < n; ++i) vn[i] /= hn;
      for (int k = 0; k < j; ++k) {                           /* old rotations */
        double a0 = H[(size_t)k * m + j], a1 = H[(size_t)(k + 1) * m + j];
        H[(size_t)k * m + j] = cs[k] * a0 + sn[k] * a1;
        H[(size_t)(k + 1) * m + j] = -sn[k] * a0 + cs[k] * a1;
      }
      double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
      double rr = sqrt(a0 * a0 + a1 * a1);
      cs[j] = (rr == 0.0) ? 1.0 : a0 / rr;
      sn[j] = (rr == 0.0) ? 0.0 : a1 / rr;
      H[(size_t)j * m + j] = rr;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      if (fabs(g[j + 1]) <= 0.5 * tol * bnorm) { ++j; break; }
    }
    for (int k = j - 1; k >= 0; --k) {                        /* back substitution */
      double acc = g[k];
      for (int l = k + 1; l < j; ++l) acc -= H[(size_t)k * m + l] * y[l];
      y[k] = acc / H[(size_t)k * m + k];
    }
    for (int i = 0; i < n; ++i) {                             /* x += D^{-1} V y */
      double acc = 0.0;
      for (int k = 0; k < j; ++k) acc += V[(size_t)k * n + i] * y[k];
      x[i] += dinv[i] * acc;
    }
  }
  if (result < 0) {
    csr_mv(n, rowptr, col, val, x, w);
    for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
    if (nrm2(n, w) <= tol * bnorm) result = total;
  }
out:
  free(dinv); free(V); free(H); free(cs); free(sn); free(g); free(y); free(w); free(t);
  return result;
}

/* ======================================================================== */
/* Metropolis chain of one walker (Sec. 2.2): particles moved in order, the  */
/* move of particle i accepted iff ratio^2 > U, U ~ U(0,1).                  */
/* ======================================================================== */
/* upper bound on the sites within r_c of any point: every site in the ball
 * owns a Voronoi cell of volume v inside the ball of radius r_c + R_cell */
static int row_capacity(const orc_system* s) {
  double rcell = s->lattice == 1 ? s->a * 0.5 * sqrt(3.0) : s->a * 0.5 * sqrt(3.0);
  double rr = s->r_c + rcell;
  double vcell = s->lattice == 1 ? 0.5 * s->a * s->a * s->a : s->a * s->a * s->a;
  double cnt = 4.0 / 3.0 * M_PI * rr * rr * rr / vcell;
  int cap = (int)cnt + 8;
  int n = orc_n(s);
  return cap < n ? cap : n;
}

long orc_chain(const orc_system* s, uint64_t seed, double sigma, int first_sweep,
               int n_sweeps, long max_steps, int solver, int refresh, double* R,
               double* ratio_log, uint8_t* accept_log, double* u_log) {
  int n = orc_n(s);
  size_t nn = (size_t)n * n;
  double* Z = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  double* rownew = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * n);
  double* A = NULL;
  double* B = NULL;
  double* work = NULL;
  /* sparse storage for solver 2: fixed-capacity row slots */
  int cap = row_capacity(s);
  int32_t* scol = NULL;
  double* sval = NULL;
  int* slen = NULL;
  int64_t* rp = NULL;
  int32_t* ci = NULL;
  double* cv = NULL;
  double* e = NULL;
  double* z = NULL;
  long steps = 0, accepted = 0;
  double L = box_len(s);
  double rc2 = s->r_c * s->r_c;
  orc_sites(s, Z);
  if (solver == 0 || solver == 1) {
    A = (double*)malloc(sizeof(double) * nn);
    orc_slater_dense(s, Z, R, A);
  }
  if (solver == 1) {
    B = (double*)malloc(sizeof(double) * nn);
    work = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    if (orc_inverse(n, A, B)) { steps = -1; goto done; }
  }
  if (solver == 2) {
    scol = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * cap);
    sval = (double*)malloc(sizeof(double) * (size_t)n * cap);
    slen = (int*)calloc((size_t)n, sizeof(int));
    rp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * cap);
    cv = (double*)malloc(sizeof(double) * (size_t)n * cap);
    e = (double*)calloc((size_t)n, sizeof(double));
    z = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) {
      int c = 0;
      for (int j = 0; j < n; ++j) {
        double v = orbital(s, Z + 3 * j, R + 3 * i, L, rc2);
        if (v != 0.0 && c < cap) { scol[(size_t)i * cap + c] = j; sval[(size_t)i * cap + c] = v; ++c; }
      }
      slen[i] = c;
    }
  }
  for (int sw = first_sweep; sw < first_sweep + n_sweeps; ++sw) {
    for (int i = 0; i < n; ++i) {
      if (max_steps >= 0 && steps >= max_steps) goto done;
      double rnew[3];
      orc_propose(s, seed, (uint32_t)sw, (uint32_t)i, sigma, R + 3 * i, rnew);
      orc_row_dense(s, Z, rnew, rownew);
      double ratio = 0.0;
      if (solver == 0 || solver == 1) {
        for (int j = 0; j < n; ++j) u[j] = rownew[j] - A[(size_t)i * n + j];
        if (solver == 0) {
          if (orc_ratio_dense(n, A, i, rownew, &ratio, NULL)) { steps = -1; goto done; }
        } else {
          ratio = orc_sm_ratio(n, B, i, u);
        }
      } else {
        for (int j = 0; j < n; ++j) u[j] = rownew[j];
        for (int c = 0; c < slen[i]; ++c) u[scol[(size_t)i * cap + c]] -= sval[(size_t)i * cap + c];
        long q = 0;
        rp[0] = 0;
        for (int r = 0; r < n; ++r) {
          for (int c = 0; c < slen[r]; ++c) {
            ci[q] = scol[(size_t)r * cap + c];
            cv[q] = sval[(size_t)r * cap + c];
            ++q;
          }
          rp[r + 1] = q;
        }
        e[i] = 1.0;
        int its = orc_gmres(n, rp, ci, cv, e, z, 200, 20000, 1e-14);
        e[i] = 0.0;
        if (its < 0) { steps = -1; goto done; }
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += u[j] * z[j];
        ratio = 1.0 + acc;
      }
      double U = orc_accept_uniform(seed, (uint32_t)sw, (uint32_t)i);
      int acc = ratio * ratio > U;
      if (ratio_log) ratio_log[steps] = ratio;
      if (accept_log) accept_log[steps] = (uint8_t)acc;
      if (u_log) u_log[steps] = U;
      if (acc) {
        for (int d = 0; d < 3; ++d) R[3 * i + d] = rnew[d];
        if (solver == 1) orc_sm_update(n, B, i, u, ratio, work);
        if (solver == 0 || solver == 1) memcpy(A + (size_t)i * n, rownew, sizeof(double) * n);
        if (solver == 2) {
          int c = 0;
          for (int j = 0; j < n; ++j)
            if (rownew[j] != 0.0 && c < cap) { scol[(size_t)i * cap + c] = j; sval[(size_t)i * cap + c] = rownew[j]; ++c; }
          slen[i] = c;
        }
        ++accepted;
        if (solver == 1 && refresh > 0 && accepted % refresh == 0)
          if (orc_inverse(n, A, B)) { steps = -1; goto done; }
      }
      ++steps;
    }
  }
done:
  free(Z); free(rownew); free(u); free(A); free(B); free(work);
  free(scol); free(sval); free(slen); free(rp); free(ci); free(cv); free(e); free(z);
  return steps;
}

long orc_chains(const orc_system* s, int n_walkers, const uint64_t* seeds, double sigma,
                int first_sweep, int n_sweeps, long max_steps, int solver, int refresh,
                double* R, double* ratio_log, uint8_t* accept_log, int threads) {
  int n = orc_n(s);
  long per = (long)n_sweeps * n;
  if (max_steps >= 0 && max_steps < per) per = max_steps;
  long total = 0;
  int failed = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) reduction(| : failed)
#endif
  for (int w = 0; w < n_walkers; ++w) {
    long st = orc_chain(s, seeds[w], sigma, first_sweep, n_sweeps, max_steps, solver, refresh,
                        R + (size_t)w * 3 * n, ratio_log ? ratio_log + (size_t)w * per : NULL,
                        accept_log ? accept_log + (size_t)w * per : NULL, NULL);
    if (st < 0) failed |= 1; else total += st;
  }
  return failed ? -1 : total;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* Geometric reordering, Sec. 3.1: the greedy particle/orbital rule.         */
/* ======================================================================== */
static double pair_dist2(const orc_system* s, const double* r, const double* z) {
  double L = box_len(s);
  double dx = min_image(r[0] - z[0], L);
  double dy = min_image(r[1] - z[1], L);
  double dz = min_image(r[2] - z[2], L);
  return dx * dx + dy * dy + dz * dz;
}

void orc_greedy_pairing(const orc_system* s, const double* R, const double* Z, int* P, int* Q) {
  int n = orc_n(s);
  for (int i = 0; i < n - 1; ++i) {
    int bj = i;
    double bd = pair_dist2(s, R + 3 * P[i], Z + 3 * Q[i]);
    for (int j = i + 1; j < n; ++j) {
      double d = pair_dist2(s, R + 3 * P[i], Z + 3 * Q[j]);
      if (d < bd) { bd = d; bj = j; }
    }
    if (bj != i) {
      int t = Q[i]; Q[i] = Q[bj]; Q[bj] = t;
    } else {
      int bk = i;
      double bdk = pair_dist2(s, R + 3 * P[i], Z + 3 * Q[i]);
      for (int k = i + 1; k < n; ++k) {
        double d = pair_dist2(s, R + 3 * P[k], Z + 3 * Q[i]);
        if (d < bdk) { bdk = d; bk = k; }
      }
      if (bk != i) { int t = P[i]; P[i] = P[bk]; P[bk] = t; }
    }
  }
}

/* ======================================================================== */
/* Kinetic energy, Eq. 21 with hbar = mass = 1.  -1/2 lap phi = (3k - 2k^2   */
/* d^2) phi for phi = exp(-k d^2), so the estimator is                       */
/*   (1/2n) sum_{p,o} (6k - 4k^2 |r_p - Z_o|^2) A_po (A^{-1})_op.            */
/* ======================================================================== */
double orc_kinetic_energy(const orc_system* s, const double* Z, const double* R) {
  int n = orc_n(s);
  size_t nn = (size_t)n * n;
  double L = box_len(s);
  double* A = (double*)malloc(sizeof(double) * nn);
  double* B = (double*)malloc(sizeof(double) * nn);
  orc_slater_dense(s, Z, R, A);
  double E = NAN;
  if (!orc_inverse(n, A, B)) {
    double acc = 0.0;
    for (int p = 0; p < n; ++p)
      for (int o = 0; o < n; ++o) {
        double apo = A[(size_t)p * n + o];
        if (apo == 0.0) continue;
        double dx = min_image(R[3 * p + 0] - Z[3 * o + 0], L);
        double dy = min_image(R[3 * p + 1] - Z[3 * o + 1], L);
        double dz = min_image(R[3 * p + 2] - Z[3 * o + 2], L);
        double d2 = dx * dx + dy * dy + dz * dz;
        acc += (6.0 * s->kappa - 4.0 * s->kappa * s->kappa * d2) * apo * B[(size_t)o * n + p];
      }
    E = acc / (2.0 * (double)n);
  }
  free(A); free(B);
  return E;
}

/* ======================================================================== */
/* Gradient and Laplacian at a proposed position (quantities of the drift   */
/* and the local energy, Sec. 2.2).  With A' = A with row i replaced by      */
/* a(r'), column i of A'^{-1} is z / ratio, z = A^{-1} e_i, so               */
/*   grad = sum_o grad phi_o(r') z_o / ratio  = grad_{r'} ln|det A'|,        */
/*   lap  = sum_o lap phi_o(r') z_o / ratio   = lap_{r'} det A' / det A',    */
/* grad phi = -2k (r - Z) phi, lap phi = (4k^2 d^2 - 6k) phi (min image).    */
/* Dense LU for z.  Returns nonzero if A is singular.                        */
/* ======================================================================== */
int orc_ratio_grad_lap(const orc_system* s, const double* Z, const double* R, int i, const double r_new[3],
                       double* ratio, double grad[3], double* lap) {
  int n = orc_n(s);
  size_t nn = (size_t)n * n;
  double L = box_len(s);
  double rc2 = s->r_c * s->r_c;
  double* A = (double*)malloc(sizeof(double) * nn);
  double* e = (double*)calloc((size_t)n, sizeof(double));
  double* z = (double*)malloc(sizeof(double) * n);
  double* a = (double*)malloc(sizeof(double) * n);
  int* piv = (int*)malloc(sizeof(int) * n);
  int sign, rc = 0;
  orc_slater_dense(s, Z, R, A);
  orc_row_dense(s, Z, r_new, a);
  {
    double acc = 0.0; /* u^T z needs the old row: take it before factoring */
    double* Acopy = (double*)malloc(sizeof(double) * nn);
    memcpy(Acopy, A, sizeof(double) * nn);
    if (orc_lu(n, A, piv, &sign)) {
      rc = 1;
    } else {
      e[i] = 1.0;
      orc_lu_solve(n, A, piv, e, z);
      for (int j = 0; j < n; ++j) acc += (a[j] - Acopy[(size_t)i * n + j]) * z[j];
      *ratio = 1.0 + acc;
      double g[3] = {0.0, 0.0, 0.0}, l = 0.0;
      for (int o = 0; o < n; ++o) {
        double dx = min_image(r_new[0] - Z[3 * o + 0], L);
        double dy = min_image(r_new[1] - Z[3 * o + 1], L);
        double dz = min_image(r_new[2] - Z[3 * o + 2], L);
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > rc2) continue;
        double ph = exp(-s->kappa * d2);
        g[0] += -2.0 * s->kappa * dx * ph * z[o];
        g[1] += -2.0 * s->kappa * dy * ph * z[o];
        g[2] += -2.0 * s->kappa * dz * ph * z[o];
        l += (4.0 * s->kappa * s->kappa * d2 - 6.0 * s->kappa) * ph * z[o];
      }
      for (int d = 0; d < 3; ++d) grad[d] = g[d] / *ratio;
      *lap = l / *ratio;
    }
    free(Acopy);
  }
  free(A); free(e); free(z); free(a); free(piv);
  return rc;
}
