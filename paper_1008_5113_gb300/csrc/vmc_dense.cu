// vmc_dense.cu -- the standard algorithm (Sec. 1) on the GPU, FP64: an explicit
// inverse B = A^{-1} per walker, the ratio 1 + u^T B e_i, and the Sherman-Morrison
// update B <- B - (B e_i)(u^T B) / ratio on acceptance, with a fresh inverse (Gauss-
// Jordan elimination with partial pivoting) every sm_refresh sweeps.  The reference
// point the sparse engines are compared with; one CTA per walker.
//
// B is row-major over (orbital, particle): the ratio reads the entries B[j][i] of the
// support of u only; the update reads the rows B[j][.] of that support and then
// streams all of B once (coalesced).  On GB300 the n^2 FP64 multiply-adds of an update
// run at the FP64 rate (about 2 per clock per SM), not at the memory rate.
#include "vmc_internal.h"
#include "vmc_geom.cuh"

namespace vmc {

// Dense A (orbital columns, particle rows) from the sparse slots into B, then
// B <- A^{-1} in place (Gauss-Jordan, partial pivoting, column swaps undone at the end).
// Returns false if a pivot is exactly zero.
__device__ bool dense_invert(const Walker& w, Shared& sh) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x, cap = w.cap;
  double* B = w.Bd;
  for (size_t idx = tid; idx < (size_t)n * n; idx += nt) B[idx] = 0.0;
  __syncthreads();
  for (int p = tid; p < n; p += nt)
    for (int t = 0; t < w.a_len[p]; ++t) B[(size_t)p * n + w.a_col[(size_t)p * cap + t]] = w.a_val[(size_t)p * cap + t];
  __syncthreads();
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    double bd = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += nt) {
      const double v = fabs(B[(size_t)i * n + k]);
      if (v > bd) { bd = v; bi = i; }
    }
    double neg = -bd;
    block_argmin(neg, bi, sh);  // largest |B[i][k]|, lowest index on ties
    const int p = bi;
    if (-neg == 0.0) { ok = false; break; }
    if (p != k)
      for (int j = tid; j < n; j += nt) {
        const double t = B[(size_t)k * n + j];
        B[(size_t)k * n + j] = B[(size_t)p * n + j];
        B[(size_t)p * n + j] = t;
      }
    if (tid == 0) w.dpiv[k] = p;
    __syncthreads();
    const double inv = 1.0 / B[(size_t)k * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      const double v = (j == k) ? inv : B[(size_t)k * n + j] * inv;
      B[(size_t)k * n + j] = v;
    }
    for (int i = tid; i < n; i += nt) w.dcol[i] = B[(size_t)i * n + k];
    __syncthreads();
    // rows i != k: B[i][j] -= f_i B[k][j] (j != k), B[i][k] = -f_i B[k][k]
    for (size_t idx = tid; idx < (size_t)n * n; idx += nt) {
      const int i = (int)(idx / n), j = (int)(idx - (size_t)i * n);
      if (i == k) continue;
      const double f = w.dcol[i];
      if (j == k) B[idx] = -f * B[(size_t)k * n + k];
      else B[idx] = fma(-f, B[(size_t)k * n + j], B[idx]);
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0 && ok; --k) {
    const int p = w.dpiv[k];
    if (p != k)
      for (int i = tid; i < n; i += nt) {
        const double t = B[(size_t)i * n + k];
        B[(size_t)i * n + k] = B[(size_t)i * n + p];
        B[(size_t)i * n + p] = t;
      }
    __syncthreads();
  }
  return ok;
}

// One Metropolis step of particle k with the explicit inverse.
__device__ void dense_step(const Walker& w, int k, uint64_t seed, uint32_t sweep, double sigma, uint8_t* acc_log,
                           double* ratio_log, Shared& sh) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x, cap = w.cap;
  Ctl* c = w.ctl;
  if (tid == 0) {
    double z[3];
    normal3(seed, sweep, (uint32_t)k, 1u, z);
    for (int d = 0; d < 3; ++d) sh.rnew[d] = wrap_box(__dadd_rn(w.R[3 * k + d], __dmul_rn(sigma, z[d])), w.L);
  }
  __syncthreads();
  if (tid < 32) {
    const int alen = build_row_warp(w, sh.rnew, sh.acol, sh.aval, cap);
    int ulen = 0;
    if (alen >= 0) ulen = build_u_warp(w, k, sh.acol, sh.aval, alen, sh.ucol, sh.uval);
    if (tid == 0) { sh.alen = alen; sh.ulen = ulen; }
  }
  __syncthreads();
  if (sh.alen < 0) {
    if (tid == 0) c->status = ST_CAPACITY;
    return;
  }
  const double* B = w.Bd;
  double part = 0.0;
  for (int t = tid; t < sh.ulen; t += nt) part += sh.uval[t] * B[(size_t)sh.ucol[t] * n + k];
  const double ratio = 1.0 + block_sum(part, sh);
  const double U = accept_uniform(seed, sweep, (uint32_t)k);
  const bool acc = __dmul_rn(ratio, ratio) > U;
  if (tid == 0) {
    if (acc_log) *acc_log = acc ? 1 : 0;
    if (ratio_log) *ratio_log = ratio;
    c->proposals += 1;
    c->accepts += acc ? 1 : 0;
  }
  if (!acc) return;
  // Sherman-Morrison: col = B e_k, row = u^T B, B -= col row^T / ratio
  for (int a = tid; a < n; a += nt) w.dcol[a] = B[(size_t)a * n + k] / ratio;
  for (int b = tid; b < n; b += nt) {
    double s = 0.0;
    for (int t = 0; t < sh.ulen; ++t) s = fma(sh.uval[t], B[(size_t)sh.ucol[t] * n + b], s);
    w.drow[b] = s;
  }
  for (int t = tid; t < sh.alen; t += nt) {
    w.a_col[(size_t)k * cap + t] = sh.acol[t];
    w.a_val[(size_t)k * cap + t] = sh.aval[t];
  }
  if (tid == 0) {
    w.a_len[k] = sh.alen;
    for (int d = 0; d < 3; ++d) w.R[3 * k + d] = sh.rnew[d];
  }
  __syncthreads();
  double* Bw = w.Bd;
  for (size_t idx = tid; idx < (size_t)n * n; idx += nt) {
    const int a = (int)(idx / n), b = (int)(idx - (size_t)a * n);
    Bw[idx] = fma(-w.dcol[a], w.drow[b], Bw[idx]);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kMaxThreads, 2) k_dense_setup(const Walker* __restrict__ W) {
  __shared__ Shared sh;
  const Walker& w = W[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int bad = 0;
  for (int p = wid; p < w.n; p += nw) {
    const int len = build_row_warp(w, w.R + 3 * p, w.a_col + (size_t)p * w.cap, w.a_val + (size_t)p * w.cap, w.cap);
    if (lane == 0) {
      if (len < 0) bad = 1;
      w.a_len[p] = len < 0 ? 0 : len;
    }
  }
  __syncthreads();
  const bool ok = dense_invert(w, sh);
  if (threadIdx.x == 0) {
    if (bad) w.ctl->status = ST_CAPACITY;
    else if (!ok) w.ctl->status = ST_BREAKDOWN;
    w.ctl->factorizations += 1;
  }
}

__global__ void __launch_bounds__(kMaxThreads, 2) k_dense_sweep(const Walker* __restrict__ W, int n_sweeps, long long sweep0,
                                                             double sigma, const uint64_t* __restrict__ seeds,
                                                             uint8_t* acc_log, double* ratio_log, int refresh) {
  __shared__ Shared sh;
  const Walker& w = W[blockIdx.x];
  const uint64_t seed = seeds[blockIdx.x];
  const int n = w.n;
  for (int s = 0; s < n_sweeps; ++s) {
    if (refresh > 0 && s > 0 && (sweep0 + s) % refresh == 0) {
      const bool ok = dense_invert(w, sh);
      if (threadIdx.x == 0) {
        w.ctl->factorizations += 1;
        if (!ok) w.ctl->status = ST_BREAKDOWN;
      }
      __syncthreads();
    }
    for (int k = 0; k < n; ++k) {
      const long long idx = (long long)n_sweeps * w.log_base + (long long)s * n + k;
      const int st = w.ctl->status;
      __syncthreads();
      if (st != ST_OK) {
        if (threadIdx.x == 0) {
          if (acc_log) acc_log[idx] = 0;
          if (ratio_log) ratio_log[idx] = 0.0;
        }
        continue;
      }
      dense_step(w, k, seed, (uint32_t)(sweep0 + s), sigma, acc_log ? acc_log + idx : nullptr,
                 ratio_log ? ratio_log + idx : nullptr, sh);
      __syncthreads();
    }
  }
}

cudaError_t launch_dense_setup(const LaunchCfg& L, const Walker* W, int nwalk) {
  k_dense_setup<<<nwalk, L.threads, 0, L.stream>>>(W);
  return cudaGetLastError();
}
cudaError_t launch_dense_sweep(const LaunchCfg& L, const Walker* W, int nwalk, int n_sweeps, long long sweep0,
                               double sigma, const uint64_t* seeds, uint8_t* acc, double* ratio, int refresh) {
  k_dense_sweep<<<nwalk, L.threads, 0, L.stream>>>(W, n_sweeps, sweep0, sigma, seeds, acc, ratio, refresh);
  return cudaGetLastError();
}

}  // namespace vmc
