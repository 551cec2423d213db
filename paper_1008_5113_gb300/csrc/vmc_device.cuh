// vmc_device.cuh -- device-side data layout and block/warp primitives of the
// sparse determinant-ratio engine (sm_103a).
//
// One walker (one independent Markov chain, Sec. 2.2) is owned by one CTA.  All of a
// walker's state lives in HBM in the layout below and stays resident across sweeps:
//   * positions R[n][3] (FP64) indexed by particle id;
//   * the Slater matrix stored BY PARTICLE in fixed-capacity slots
//     (a_col/a_val[p*cap + t], a_len[p]) so that accepting a move rewrites one slot
//     (Sec. 3 Eq. 11) and a reordering (Sec. 3.1) moves no matrix data: the row of
//     the reordered matrix A_p = P A Q0 at position r is slot part_of_row[r];
//   * column labels are "positions": orbital o sits in the fixed column col_of_orb[o]
//     (orbitals laid out by a 27-colouring of their lattice site, which keeps the
//     triangular-solve dependency depth small; see vmc_layout.cpp);
//   * ILUTP factors of A_p Q = L U (Sec. 3.2 Eq. 14) in fixed-capacity rows, the
//     column permutation perm/iperm, and level sets for the triangular solves;
//   * the chain of rank-one preconditioner updates (z_hat_s, u_s) of Sec. 3.2 Eq. 18
//     with the small matrix G[s][t] = u_s^T z_hat_t;
//   * the Krylov basis V and preconditioned vectors Zk of GMRES (Sec. 3.2 Eq. 15).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vmc {

constexpr int kMaxThreads = 512;  // largest walker CTA
constexpr int kMaxM = 40;         // largest Krylov dimension
constexpr int kMaxRow = 256;      // largest Slater row (entries)
constexpr int kMaxU = 2 * kMaxRow;
constexpr int kMaxRowNZ = 2048;   // ILUTP working-row entries before dropping
constexpr int kMaxSel = 1024;     // ILUTP candidates of one triangle
constexpr int kMaxUpd = 128;      // longest preconditioner update chain
constexpr int kHistBins = 64;

// status codes (mirror vmc_status)
enum : int {
  ST_OK = 0, ST_INVALID = 1, ST_CUDA = 2, ST_OOM = 3, ST_NOCONV = 4,
  ST_BREAKDOWN = 5, ST_TIMEOUT = 6, ST_STATE = 7, ST_CAPACITY = 8
};

// Mutable per-walker controller state and statistics (device resident).
struct Ctl {
  int nlev_l, nlev_u;
  int n_upd;
  int p_lfil;
  int status;
  int pend_valid, pend_k, pend_alen, pend_ulen;
  int last_pivots;
  int last_breakdown;
  double pend_r[3];
  double pend_ratio;
  double its_sum;
  long long its_cnt;
  long long proposals, accepts, solves, inner_its, first_its, outer_passes;
  long long reorders, reorder_monitor, reorder_noconv, reorder_slow, reorder_breakdown;
  long long refactors_updates, factorizations;
  double N_max_seen, N_sum;
  double nnz_A, nnz_LU;
  long long hist[kHistBins];
};

// Immutable-per-context description of one walker: sizes and device pointers.
struct Walker {
  int n, K, lattice, cap, capLU, m, mu;
  int per;                // sites per cubic cell (1 sc, 2 bcc)
  double a, kappa, rc, rc2, L;
  const double* Z;        // n*3 orbital centres
  const int* col_of_orb;  // fixed column of each orbital
  const int* orb_of_col;
  double* R;              // n*3 positions by particle
  int* row_of_part;
  int* part_of_row;
  int* a_col; double* a_val; float* a_val32; int* a_len;
  int* l_col; double* l_val64; void* l_valT; int* l_len;
  int* u_col; double* u_val64; void* u_valT; int* u_len;
  double* u_dinv64; void* u_dinvT;
  int* perm; int* iperm;
  int* lev_l; int* lev_u;
  int* l_lvl_ptr; int* l_lvl_rows; int* u_lvl_ptr; int* u_lvl_rows; int* lvl_cur;
  double* wrow; int* wpos; int* gP; int* gQ;
  void* upd_z; int* upd_ucol; void* upd_uval; int* upd_ulen; double* upd_G;
  void* V; void* Zk; void* tv;
  double* x64; double* r64;
  int* pend_acol; double* pend_aval; int* pend_ucol; double* pend_uval;
  Ctl* ctl;
  long long log_base;     // first log entry of this walker for one sweep (prefix of n)
};

struct Params {
  double drop_tol, permtol;
  int lfil_extra, m, max_restarts, max_updates;
  double inner_rtol, ratio_tol, N_max, slow_factor;
};

// Shared memory of a walker CTA (static, < 48 KB).
struct __align__(16) Shared {
  double H[(kMaxM + 1) * kMaxM];
  double g[kMaxM + 1], cs[kMaxM], sn[kMaxM], y[kMaxM];
  double h1[kMaxM + 2], h2[kMaxM + 2];
  double red[40];
  double redv[33];
  int redi[33];
  double rnew[3];
  double aval[kMaxRow];
  int acol[kMaxRow];
  double uval[kMaxU];
  int ucol[kMaxU];
  int nz[kMaxRowNZ];
  int selF[kMaxSel];
  double selV[kMaxSel];
  double cupd[kMaxUpd];
  int alen, ulen;
  int iflag[8];
  double dflag[8];
};

// ---- warp / block reductions (fixed butterfly order: deterministic) ----------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_int(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_int(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block sum of one double; every thread gets the result.
__device__ __forceinline__ double block_sum(double v, Shared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh.redv[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < nw ? sh.redv[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh.redv[32] = t;
  }
  __syncthreads();
  double r = sh.redv[32];
  __syncthreads();
  return r;
}

// Block max of one int; every thread gets the result.
__device__ __forceinline__ int block_max_int(int v, Shared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max_int(v);
  if (lane == 0) sh.redi[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? sh.redi[lane] : -0x7fffffff;
    t = warp_max_int(t);
    if (lane == 0) sh.redi[32] = t;
  }
  __syncthreads();
  const int r = sh.redi[32];
  __syncthreads();
  return r;
}

// Block argmin of (d, j) in lexicographic order; every thread gets (d, j).
__device__ __forceinline__ void block_argmin(double& d, int& j, Shared& sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    double d2 = __shfl_xor_sync(0xffffffffu, d, o);
    int j2 = __shfl_xor_sync(0xffffffffu, j, o);
    if (d2 < d || (d2 == d && j2 < j)) { d = d2; j = j2; }
  }
  if (lane == 0) { sh.redv[wid] = d; sh.redi[wid] = j; }
  __syncthreads();
  if (wid == 0) {
    double dd = lane < nw ? sh.redv[lane] : 1e300;
    int jj = lane < nw ? sh.redi[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      double d2 = __shfl_xor_sync(0xffffffffu, dd, o);
      int j2 = __shfl_xor_sync(0xffffffffu, jj, o);
      if (d2 < dd || (d2 == dd && j2 < jj)) { dd = d2; jj = j2; }
    }
    if (lane == 0) { sh.redv[32] = dd; sh.redi[32] = jj; }
  }
  __syncthreads();
  d = sh.redv[32];
  j = sh.redi[32];
  __syncthreads();
}

}  // namespace vmc
