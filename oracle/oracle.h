/*
 * oracle.h -- plain, slow, FP64 CPU oracle for the sparse-VMC determinant ratio.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this library: only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only through the seeded workload parameters.
 *
 * What it computes (Ahuja, Clark, de Sturler, Ceperley, Kim, "Improved Scaling
 * for Quantum Monte Carlo on Insulators"):
 *   - Slater matrix a_ij = phi_j(r_i)                                (Eq. 2, Sec. 2.1)
 *   - Gaussian orbitals phi_j(r) = exp(-k |r - Z_j|^2), truncated     (Eq. 3, Sec. 2.1)
 *   - single-particle Metropolis moves, accept if ratio^2 > U(0,1)   (Sec. 2.2)
 *   - row update u_j = phi_j(r') - phi_j(r_i)                         (Eq. 12, Sec. 3)
 *   - det ratio = 1 + u^T A^{-1} e_i                                   (Eq. 2 of Sec. 1 / Eq. 13, Sec. 3)
 *   - the standard algorithm: explicit inverse + Sherman-Morrison      (Sec. 1)
 *   - kinetic-energy estimator                                         (Eq. 21, Sec. 4)
 *   - gradient and Laplacian of det at a proposed position             (Sec. 2.2)
 * The random numbers are Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * written here from its published definition, with Box-Muller normals.
 *
 * The oracle does NOT model ILUTP, the preconditioner updates, the reordering or
 * the stability monitor: those change the cost of a solve, not its result, which
 * is the exact ratio up to the solver tolerance.
 */
#ifndef VMC_ORACLE_H
#define VMC_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int K;          /* lattice cells per box side                                  */
  int lattice;    /* 0 = simple cubic (n = K^3), 1 = body-centred cubic (2 K^3)  */
  double a;       /* lattice constant; the periodic box side is L = K a          */
  double kappa;   /* Gaussian decay rate "k" of Eq. 3                            */
  double r_c;     /* cutoff: phi_j(r) = 0 when the min-image |r - Z_j| > r_c     */
} orc_system;

/* ---- counter-based RNG (Salmon et al. SC'11) ---------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* uniform in the open interval (0,1) from two 32-bit words: (top52 + 1/2) 2^-52 */
double orc_uniform53(uint32_t hi, uint32_t lo);
/* three N(0,1) normals for (seed, sweep, particle, purpose) via Box-Muller */
void orc_normal3(uint64_t seed, uint32_t sweep, uint32_t particle, uint32_t purpose,
                 double z[3]);
/* the Metropolis uniform U for (seed, sweep, particle) (purpose 2) */
double orc_accept_uniform(uint64_t seed, uint32_t sweep, uint32_t particle);

/* ---- geometry ----------------------------------------------------------------- */
int orc_n(const orc_system* s);
void orc_sites(const orc_system* s, double* Z /* n*3 */);
/* positions r_i = wrap(Z_i + jitter * N(0,1)^3), purpose 0, sweep 0 */
void orc_initial_positions(const orc_system* s, uint64_t seed, double jitter, double* R);
/* proposal r' = wrap(r + sigma * N(0,1)^3), purpose 1 */
void orc_propose(const orc_system* s, uint64_t seed, uint32_t sweep, uint32_t particle,
                 double sigma, const double r_old[3], double r_new[3]);
/* dense orbital row a_j = phi_j(r), j = 0..n-1 */
void orc_row_dense(const orc_system* s, const double* Z, const double r[3], double* row);
/* dense Slater matrix, row-major n*n */
void orc_slater_dense(const orc_system* s, const double* Z, const double* R, double* A);
/* Slater matrix in CSR (column indices ascending); returns nnz, or -1 if cap too small */
long orc_slater_csr(const orc_system* s, const double* Z, const double* R, long cap,
                    int64_t* rowptr, int32_t* col, double* val);

/* ---- dense linear algebra ----------------------------------------------------- */
/* LU with partial pivoting, in place, row-major; returns 0, or 1 if exactly singular */
int orc_lu(int n, double* A, int* piv, int* sign);
void orc_lu_solve(int n, const double* LU, const int* piv, const double* b, double* x);
/* log|det A| and sign(det A) from an LU factorisation */
double orc_lu_logabsdet(int n, const double* LU, int sign, int* det_sign);
/* Leibniz permutation sum, n <= 9 (exact definition of the determinant) */
double orc_leibniz_det(int n, const double* A);
/* ratio det(A')/det(A), A' = A with row i replaced by a_new:
 *   ratio = 1 + u^T z with A z = e_i (dense LU solve), u = a_new - A[i,:];
 *   *ratio_logdet = sign' sign exp(log|det A'| - log|det A|) (independent check). */
int orc_ratio_dense(int n, const double* A, int i, const double* a_new, double* ratio,
                    double* ratio_logdet);
/* explicit inverse via LU (B = A^{-1}, row-major) */
int orc_inverse(int n, const double* A, double* B);
/* standard algorithm: ratio from the inverse, and the Sherman-Morrison update */
double orc_sm_ratio(int n, const double* B, int i, const double* u);
void orc_sm_update(int n, double* B, int i, const double* u, double ratio, double* work);

/* ---- sparse reference solve (n > 1000): restarted GMRES, Jacobi-scaled -------- */
/* Solves A x = b to ||b - A x||_2 <= tol ||b||_2; returns iterations or -1. */
int orc_gmres(int n, const int64_t* rowptr, const int32_t* col, const double* val,
              const double* b, double* x, int restart, int max_iter, double tol);

/* ---- Metropolis chain of one walker (independent mode) ------------------------ */
/* solver: 0 = dense LU per step (the definition), 1 = explicit inverse +
 * Sherman-Morrison with a fresh inverse every refresh accepted moves,
 * 2 = sparse GMRES per step.  Runs n_sweeps sweeps of n moves in particle order,
 * starting at sweep index first_sweep, stopping after max_steps moves if
 * max_steps >= 0.  R (n*3) holds the start positions and receives the final ones.
 * Logs (nullable, one entry per move): ratio, accept (0/1), U.
 * Returns the number of moves made, or -1 on a singular matrix. */
long orc_chain(const orc_system* s, uint64_t seed, double sigma, int first_sweep,
               int n_sweeps, long max_steps, int solver, int refresh, double* R,
               double* ratio_log, uint8_t* accept_log, double* u_log);
/* several independent walkers, OpenMP across walkers (threads = 0: default) */
long orc_chains(const orc_system* s, int n_walkers, const uint64_t* seeds, double sigma,
                int first_sweep, int n_sweeps, long max_steps, int solver, int refresh,
                double* R /* n_walkers*n*3 */, double* ratio_log /* n_walkers*steps */,
                uint8_t* accept_log, int threads);
int orc_max_threads(void);

/* ---- geometric reordering (Sec. 3.1, the greedy rule) -------------------------- */
/* P[i] = particle at position i, Q[i] = orbital at position i (in/out).  For
 * i = 0..n-2: the orbital nearest to particle P[i] among positions >= i is swapped into
 * position i; if that is already position i, the particle nearest to orbital Q[i] among
 * positions >= i is swapped into position i.  Minimum-image distances, ties to the
 * lowest position. */
void orc_greedy_pairing(const orc_system* s, const double* R, const double* Z, int* P, int* Q);

/* ---- kinetic energy (Eq. 21): (1/2n) sum_{p,o} (6k - 4k^2 |r_p - Z_o|^2) A_po (A^-1)_op */
double orc_kinetic_energy(const orc_system* s, const double* Z, const double* R);

/* ---- gradient and Laplacian at a proposed position (drift and local energy, Sec. 2.2):
 * ratio as orc_ratio_dense; grad = grad_{r'} ln|det A'|, lap = lap_{r'} det A' / det A',
 * A' = A with row i replaced by the row at r_new.  Nonzero return: A singular. */
int orc_ratio_grad_lap(const orc_system* s, const double* Z, const double* R, int i, const double r_new[3],
                       double* ratio, double grad[3], double* lap);

#ifdef __cplusplus
}
#endif
#endif
