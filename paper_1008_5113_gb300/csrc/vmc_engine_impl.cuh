// vmc_engine_impl.cuh -- the templated kernels of the sparse determinant-ratio engine and
// their launchers, instantiated once per working precision (vmc_engine_f64.cu,
// vmc_engine_f32.cu) so that the two precisions compile in parallel.
//
// Every kernel runs one CTA per walker, except k_sweep_pair: a cluster of two CTAs per
// walker, the second refactoring in the background (see the section below).  Besides
// the sweeps: the single-move calls (k_ratio, with the drift quantities on request;
// k_accept), the kinetic energy (k_kinetic), set-up and inspection kernels.
// A Metropolis step (Sec. 2.2) is:
//   propose r' (Philox, purpose 1) -> Slater row a' and u = a' - a_k (Sec. 3 Eq. 12)
//   -> solve A_p x = e_r by preconditioned GMRES (Sec. 3.2 Eq. 15) with FP64 refinement
//   -> controller: reorder + refactor when N > N_max, GMRES fails to converge in m
//      iterations, or the iterations reach slow_factor x the running average (Sec. 4)
//   -> ratio 1 + u^T x (Sec. 3 Eq. 13), accept iff ratio^2 > U (Sec. 2.2)
//   -> on accept: replace the row and push (z_hat = x / ratio, u) onto the update
//      chain (Sec. 3.2 Eq. 17); a new ILUTP once the chain holds max_updates entries
//      (Sec. 3.2, last paragraph).
#pragma once
#include "vmc_internal.h"
#include "vmc_krylov.cuh"

namespace vmc {


// ---------------------------------------------------------------------------
// device: solve + controller for the move in shared memory (sh.acol/aval, sh.ucol/uval)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ void solve_with_controller(const Walker& w, const Params& P, int k, SolveOut& o, Shared& sh) {
  // The solve of the move runs to completion first: GMRES cycles restart from the FP64
  // residual until the ratio reaches its accuracy goal, so no trigger can leave the
  // ratio inaccurate.  The controller then judges the preconditioner by the paper's
  // three tests (Sec. 4): the stability monitor N > N_max over the Arnoldi vectors of
  // the first cycle; GMRES not reaching the tolerance trig_rtol (1e-6) within the
  // maximum iteration count trig_its (40); the iterations to that tolerance reaching
  // slow_factor (4) x the running average.  Any of them reorders (Sec. 3.1) and
  // refactors now, for the moves that follow.
  Ctl* c = w.ctl;
  const double rtol = P.inner_rtol;
  const int brow = w.row_of_part[k];
  long long t0 = clock64();
  solve_first<T>(w, P, brow, rtol, o, sh);
  if (threadIdx.x == 0) c->cyc[PH_FIRST] += clock64() - t0;
  t0 = clock64();
  refine<T>(w, P, brow, rtol, 2 + P.max_restarts, o, sh);
  if (threadIdx.x == 0) c->cyc[PH_REFINE] += clock64() - t0;
  if (o.status == ST_NOCONV && !c->fresh) {
    // out of cycles: reorder, refactor and solve again from scratch (Sec. 4)
    const int fl = factor_block<T>(w, P, sh, true);
    if (threadIdx.x == 0) {
      c->reorders += 1;
      c->reorder_noconv += 1;
      c->inner_its += o.total_its;
      c->solves += 1;
      if (fl & 2) c->status = ST_CAPACITY;
    }
    __syncthreads();
    const int brow2 = w.row_of_part[k];
    t0 = clock64();
    solve_first<T>(w, P, brow2, rtol, o, sh);
    refine<T>(w, P, brow2, rtol, 4 * (2 + P.max_restarts), o, sh);  // and allow more cycles
    if (threadIdx.x == 0) c->cyc[PH_REFINE] += clock64() - t0;
  }
  const int kits = o.its_trig >= 0 ? o.its_trig : o.total_its;  // iterations to the tolerance
  int cause = 0;
  const long long cnt = c->its_cnt;
  const double avg = cnt > 0 ? c->its_sum / (double)cnt : 0.0;
  if (o.its_trig < 0 || o.its_trig > P.trig_its) cause = 2;
  else if (o.N > P.N_max) cause = 1;
  else if (cnt >= 10 && (double)kits >= P.slow_factor * avg) cause = 3;
  // A reorder + refactorisation of a matrix that has not changed since the last one
  // reproduces the same factors (both are deterministic): it is skipped.
  const bool skip = cause != 0 && c->fresh != 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (sh.iflag[3] && c->status == ST_OK) c->status = ST_TIMEOUT;
    c->solves += 1;
    c->inner_its += o.total_its;
    c->first_its += o.its1;
    c->trig_its += kits;
    c->outer_passes += o.passes;
    c->N_max_seen = fmax(c->N_max_seen, o.N);
    c->N_sum += o.N;
    c->hist[min(o.its1, kHistBins - 1)] += 1;
    if (o.status != ST_OK && c->status == ST_OK) c->status = o.status;
    if (skip) c->reorder_skipped += 1;
    if (!cause || skip) {
      c->its_sum += (double)kits;
      c->its_cnt += 1;
    }
  }
  __syncthreads();
  if (cause && !skip && o.status == ST_OK) {
    const int fl = factor_block<T>(w, P, sh, true);
    if (threadIdx.x == 0) {
      c->reorders += 1;
      if (cause == 1) c->reorder_monitor += 1;
      if (cause == 2) c->reorder_noconv += 1;
      if (cause == 3) c->reorder_slow += 1;
      if (fl & 2) c->status = ST_CAPACITY;
    }
  }
  __syncthreads();
}

// Commit the move in shared memory for particle k (row replace + preconditioner update).
template <typename T>
__device__ __noinline__ void commit_move(const Walker& w, const Params& P, int k, double ratio, Shared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x, n = w.n, cap = w.cap;
  const int alen = sh.alen, ulen = sh.ulen;
  const long long t0 = clock64();
  for (int t = tid; t < alen; t += nt) {
    w.a_col[(size_t)k * cap + t] = sh.acol[t];
    w.a_val[(size_t)k * cap + t] = sh.aval[t];
    w.a_val32[(size_t)k * cap + t] = (float)sh.aval[t];
  }
  if (tid == 0) {
    w.ctl->fresh = 0;
    w.a_len[k] = alen;
    w.R[3 * k] = sh.rnew[0];
    w.R[3 * k + 1] = sh.rnew[1];
    w.R[3 * k + 2] = sh.rnew[2];
  }
  Ctl* c = w.ctl;
  const int s = c->n_upd;
  __syncthreads();
  if (s < P.max_updates) {
    T* Zh = (T*)w.upd_z;
    T* Uv = (T*)w.upd_uval;
    const double inv = 1.0 / ratio;
    for (int i = tid; i < n; i += nt) Zh[(size_t)i * w.mu4 + s] = (T)(w.x64[i] * inv);  // transposed
    for (int t = tid; t < ulen; t += nt) {
      w.upd_ucol[(size_t)s * kMaxU + t] = sh.ucol[t];
      Uv[(size_t)s * kMaxU + t] = (T)sh.uval[t];
    }
    if (tid == 0) { w.upd_ulen[s] = ulen; c->upd_nnz += ulen; }
    __syncthreads();
    // G[s][t] = u_s^T z_hat_t for t < s, from the stored (working-precision) values
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int t = wid; t < s; t += nw) {
      double acc = 0.0;
      for (int e = lane; e < ulen; e += 32)
        acc += (double)Uv[(size_t)s * kMaxU + e] * (double)Zh[(size_t)w.upd_ucol[(size_t)s * kMaxU + e] * w.mu4 + t];
      acc = warp_sum(acc);
      if (lane == 0) w.upd_G[(size_t)s * kMaxUpd + t] = acc;
    }
    __syncthreads();
    if (tid == 0) c->n_upd = s + 1;
  } else {
    int fl = factor_block<T>(w, P, sh, false);
    if (tid == 0) c->refactors_updates += 1;
    if (fl & 1) {
      fl = factor_block<T>(w, P, sh, true);
      if (tid == 0) { c->reorders += 1; c->reorder_breakdown += 1; }
    }
    if (tid == 0 && (fl & 2)) c->status = ST_CAPACITY;
  }
  if (tid == 0) c->cyc[PH_COMMIT] += clock64() - t0;
  __syncthreads();
}

// Build a' for the particle k at sh.rnew and u = a' - a_k (warp 0).  Returns false on
// a capacity overflow (status set).
static __device__ __noinline__ bool build_move(const Walker& w, int k, Shared& sh) {
  if (threadIdx.x < 32) {
    const int alen = build_row_warp(w, sh.rnew, sh.acol, sh.aval, w.cap);
    int ulen = 0;
    if (alen >= 0) ulen = build_u_warp(w, k, sh.acol, sh.aval, alen, sh.ucol, sh.uval);
    if (threadIdx.x == 0) { sh.alen = alen; sh.ulen = ulen; }
  }
  __syncthreads();
  if (sh.alen < 0) {
    if (threadIdx.x == 0) w.ctl->status = ST_CAPACITY;
    __syncthreads();
    return false;
  }
  return true;
}

// One Metropolis step of particle k (Sec. 2.2).
template <typename T>
__device__ __noinline__ void mc_step(const Walker& w, const Params& P, int k, uint64_t seed, uint32_t sweep, double sigma,
                        uint8_t* acc_log, double* ratio_log, Shared& sh) {
  Ctl* c = w.ctl;
  const int st = c->status;
  __syncthreads();
  if (st != ST_OK) {
    if (threadIdx.x == 0) {
      if (acc_log) *acc_log = 0;
      if (ratio_log) *ratio_log = 0.0;
    }
    return;
  }
  const long long t_step = clock64();
  if (threadIdx.x == 0) {
    double z[3];
    normal3(seed, sweep, (uint32_t)k, 1u, z);
    for (int d = 0; d < 3; ++d) sh.rnew[d] = wrap_box(__dadd_rn(w.R[3 * k + d], __dmul_rn(sigma, z[d])), w.L);
  }
  __syncthreads();
  if (!build_move(w, k, sh)) return;
  if (threadIdx.x == 0) c->cyc[PH_BUILD] += clock64() - t_step;
  SolveOut o;
  solve_with_controller<T>(w, P, k, o, sh);
  const double U = accept_uniform(seed, sweep, (uint32_t)k);
  const bool ok = o.status == ST_OK;
  const bool acc = ok && __dmul_rn(o.ratio, o.ratio) > U;
  if (threadIdx.x == 0) {
    if (acc_log) *acc_log = acc ? 1 : 0;
    if (ratio_log) *ratio_log = o.ratio;
    c->proposals += 1;
    c->accepts += acc ? 1 : 0;
  }
  if (acc) commit_move<T>(w, P, k, o.ratio, sh);
  if (threadIdx.x == 0) c->cyc[PH_STEP] += clock64() - t_step;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Background refactorisation (k_sweep_pair).  The second CTA of a walker's cluster
// factors a snapshot of A while the first keeps stepping, and the solver then re-roots
// the update chain on the new factors.  With U_s = I - z_hat_s u_s^T the identity
// A_{s+1} M_{s+1} = A_s M_s (Sec. 3.2 Eqs. 16-18) holds whatever M the chain starts
// from, so after the swap the solver applies U_{m-1} ... U_{s0} (LU of A_{s0})^{-1} and
// drops the updates older than the snapshot s0.  The factor CTA may also re-pair
// particles and orbitals first (greedy reordering, Sec. 3.1): a new row order P' leaves
// x = A_p^{-1} e_{row(k)}, z_hat and u (column space) unchanged, so the chain carries
// over to the re-paired root as well.  A snapshot is taken when the chain
// holds af_lag updates past its root and its factors are adopted exactly af_lag accepts
// later (waiting for them if need be), so the preconditioner sequence -- and every
// result -- is independent of how fast the factor CTA runs.
// ---------------------------------------------------------------------------

// Thread 0: move the factor CTA's statistics into the solver's controller.
static __device__ void af_take_stats(Ctl* c, Ctl* sc) {
  c->factorizations += sc->factorizations; sc->factorizations = 0;
  c->cyc[PH_ILUTP] += sc->cyc[PH_ILUTP]; sc->cyc[PH_ILUTP] = 0;
  c->cyc[PH_LEVELS] += sc->cyc[PH_LEVELS]; sc->cyc[PH_LEVELS] = 0;
  c->af_factor_cyc += sc->cyc[PH_FACTOR]; sc->cyc[PH_FACTOR] = 0;
  c->ilu_rows += sc->ilu_rows; sc->ilu_rows = 0;
  c->ilu_elims += sc->ilu_elims; sc->ilu_elims = 0;
  c->ilu_cand += sc->ilu_cand; sc->ilu_cand = 0;
}

// Block-wide: adopt factor set af_target and keep the chain entries s0 .. n_upd - 1
// (moved to 0 .. n_upd - 1 - s0; G[s][t] = u_s^T z_hat_t does not depend on the root).
template <typename T>
__device__ void af_swap(const Walker& w0, const Params& P, Shared& sh) {
  Ctl* c = w0.ctl;
  const Ctl* sc = w0.shadow;
  const int tid = threadIdx.x, nt = blockDim.x, n = w0.n;
  const int s0 = c->af_snap, len = c->n_upd - s0;
  T* Zt = (T*)w0.upd_z;
  const int mcap = w0.mu4;
  for (int i = tid; i < n; i += nt) {
    T* zr = Zt + (size_t)i * mcap;
    for (int j = 0; j < len; ++j) zr[j] = zr[s0 + j];
  }
  T* Uv = (T*)w0.upd_uval;
  for (int j = 0; j < len; ++j) {  // destination rows in increasing order: sources are intact
    const int ul = w0.upd_ulen[s0 + j];
    for (int t = tid; t < ul; t += nt) {
      w0.upd_ucol[(size_t)j * kMaxU + t] = w0.upd_ucol[(size_t)(s0 + j) * kMaxU + t];
      Uv[(size_t)j * kMaxU + t] = Uv[(size_t)(s0 + j) * kMaxU + t];
    }
    for (int t = tid; t < j; t += nt) w0.upd_G[(size_t)j * kMaxUpd + t] = w0.upd_G[(size_t)(s0 + j) * kMaxUpd + s0 + t];
    __syncthreads();
    if (tid == 0) w0.upd_ulen[j] = ul;
  }
  if (P.af_reorder) {
    // the new row pairing comes with the factors; the chain lives in column space and
    // x = A_p^{-1} e_{row(k)} does not depend on the row order, so it carries over
    for (int r = tid; r < n; r += nt) {
      w0.part_of_row[r] = w0.snap_part[r];
      w0.row_of_part[r] = w0.snap_rop[r];
    }
  }
  __syncthreads();
  if (tid == 0) {
    int nnzu = 0;
    for (int j = 0; j < len; ++j) nnzu += w0.upd_ulen[j];
    c->upd_nnz = nnzu;
    c->n_upd = len;
    c->nlev_l = sc->nlev_l; c->nlev_u = sc->nlev_u;
    c->ngrp_l = sc->ngrp_l; c->ngrp_u = sc->ngrp_u;
    c->nchunk_l = sc->nchunk_l; c->nchunk_u = sc->nchunk_u;
    c->stream_bytes = sc->stream_bytes;
    c->nnz_LU = sc->nnz_LU; c->nnz_A = sc->nnz_A;
    c->p_lfil = sc->p_lfil; c->last_pivots = sc->last_pivots; c->last_breakdown = 0;
    c->active = c->af_target;
    c->fresh = 0;
    c->refactors_async += 1;
    st_release(&c->af_state, 0);
  }
  fence_proxy_async_global();  // the new streams are read by bulk copies next
  __syncthreads();
}

// Block-wide, before every step of the solver CTA: adopt finished factors when the
// chain has reached snapshot + af_lag, and request the next factorisation.
template <typename T>
__device__ __noinline__ void af_step_begin(const Walker& w0, const Params& P, Shared& sh) {
  Ctl* c = w0.ctl;
  if (threadIdx.x == 0) {
    int act = 0;  // 1 adopt, 2 reorder + refactor now (the background one broke down)
    const long long t0 = clock64();
    int st = ld_acquire(&c->af_state);
    const int nu = c->n_upd;
    if (st != 0 && c->af_epoch_req != c->af_epoch) {
      // stale: a synchronous factorisation came after the snapshot; wait for it (only
      // when a new request is due, so that the request point stays fixed) and drop it
      if (st == 1 && nu >= P.af_lag) st = wait_state_change(&c->af_state, 1);
      if (st == 2) {
        af_take_stats(c, w0.shadow);
        st_release(&c->af_state, 0);
      }
    } else if (st != 0 && nu >= c->af_snap + P.af_lag) {
      if (st == 1) st = wait_state_change(&c->af_state, 1);
      if (st == 2) {
        af_take_stats(c, w0.shadow);
        const int fl = c->af_fail;
        if (fl & 2) {
          c->status = ST_CAPACITY;
          st_release(&c->af_state, 0);
        } else if (fl & 1) {
          act = 2;
          st_release(&c->af_state, 0);
        } else {
          act = 1;
        }
      }
    }
    if (st < 0 && c->status == ST_OK) c->status = ST_TIMEOUT;
    c->af_wait_cyc += clock64() - t0;
    sh.iflag[4] = act;
  }
  __syncthreads();
  const int act = sh.iflag[4];
  if (act == 1) {
    fence_acq_rel_gpu();
    af_swap<T>(w0, P, sh);
  } else if (act == 2) {
    const int fl = factor_block<T>(active_of(w0), P, sh, true);
    if (threadIdx.x == 0) {
      c->reorders += 1;
      c->reorder_breakdown += 1;
      if (fl & 2) c->status = ST_CAPACITY;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    sh.iflag[7] = (c->status == ST_OK && ld_acquire(&c->af_state) == 0 && c->n_upd >= P.af_lag) ? 1 : 0;
  __syncthreads();
  if (sh.iflag[7]) {
    const int n = w0.n, tid = threadIdx.x, nt = blockDim.x;
    for (size_t idx = tid; idx < (size_t)n * w0.cap; idx += nt) {
      w0.snap_col[idx] = w0.a_col[idx];
      w0.snap_val[idx] = w0.a_val[idx];
    }
    for (int p = tid; p < n; p += nt) {
      w0.snap_len[p] = w0.a_len[p];
      w0.snap_part[p] = w0.part_of_row[p];
    }
    if (P.af_reorder)
      for (int i = tid; i < 3 * n; i += nt) w0.snap_R[i] = w0.R[i];
    __syncthreads();
    if (tid == 0) {
      c->af_snap = c->n_upd;
      c->af_epoch_req = c->af_epoch;
      c->af_target = 1 - c->active;
      __threadfence();
      st_release(&c->af_state, 1);
    }
  }
  __syncthreads();
}

// Thread 0 of the solver CTA, at the end of a launch: let the factor CTA finish the
// request in flight, then tell it to leave.
static __device__ void af_finish(const Walker& w0, int launch_id) {
  Ctl* c = w0.ctl;
  int st = ld_acquire(&c->af_state);
  if (st == 1) st = wait_state_change(&c->af_state, 1);
  if (st < 0 && c->status == ST_OK) c->status = ST_TIMEOUT;
  st_release(&c->af_stop, launch_id);
}

// The factor CTA: serve requests until the solver CTA marks the end of the launch.
template <typename T>
__device__ __noinline__ void af_factor_loop(const Walker& w0, const Params& P, int launch_id, Shared& sh) {
  Ctl* c = w0.ctl;
  for (;;) {
    if (threadIdx.x == 0) {
      int r = 3;  // 1 work, 2 stop, 3 gave up waiting
      const unsigned long long t0 = global_ns();
      for (;;) {
        if (ld_acquire(&c->af_state) == 1) { r = 1; break; }
        if (ld_acquire(&c->af_stop) == launch_id) { r = 2; break; }
        if (global_ns() - t0 > kPairWaitNs) break;
        __nanosleep(2000);
      }
      sh.iflag[5] = r;
      sh.iflag[6] = r == 1 ? c->af_target : 0;
    }
    __syncthreads();
    if (sh.iflag[5] != 1) break;  // the solver's own bounded waits report a lost partner
    fence_acq_rel_gpu();
    const Walker& wf = *w0.fact[sh.iflag[6]];
    const int fl = factor_block<T>(wf, P, sh, P.af_reorder != 0);
    __syncthreads();
    if (threadIdx.x == 0) {
      c->af_fail = fl & 3;
      __threadfence();
      st_release(&c->af_state, 2);
    }
    __syncthreads();
  }
}

// Budgeted advance (block-wide): the walker claims moves one at a time from the batch's
// budget and makes them along its own chain -- particle pos_k of sweep pos_sweep onwards
// -- so that walkers whose solves are cheaper make more moves and no SM idles while the
// slowest walker finishes a fixed share.  Each walker's chain is the one fixed sweeps
// give (the proposals and uniforms are keyed by sweep and particle, and the factor
// adoption points by accept counts); only the number of moves each walker makes in one
// launch depends on timing.
template <typename T, bool PAIR>
__device__ void advance_budget(const Walker& w0, const Params& P, long long sweep0, double sigma, uint64_t seed,
                               Shared& sh) {
  Ctl* c = w0.ctl;
  const int n = w0.n, lim = P.step_limit > 0 ? min(n, P.step_limit) : n;
  long long sw = c->pos_valid ? c->pos_sweep : sweep0;
  int k = c->pos_valid ? c->pos_k : 0;
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0)
      sh.iflag[9] = atomicAdd(P.budget_ctr, 1ull) < (unsigned long long)P.budget_total ? 1 : 0;
    __syncthreads();
    const int go = sh.iflag[9];
    __syncthreads();
    if (!go) break;
    if (PAIR) af_step_begin<T>(w0, P, sh);
    mc_step<T>(active_of(w0), P, k, seed, (uint32_t)sw, sigma, nullptr, nullptr, sh);
    if (++k == lim) { k = 0; ++sw; }
  }
  if (threadIdx.x == 0) { c->pos_sweep = sw; c->pos_k = k; c->pos_valid = 1; }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_sweep(const Walker* __restrict__ W, int walker0, Params P, int n_sweeps,
                                                long long sweep0, double sigma, const uint64_t* __restrict__ seeds,
                                                uint8_t* acc_log, double* ratio_log) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const int wi = walker0 + blockIdx.x;
  const Walker& w = active_of(W[wi]);
  const uint64_t seed = seeds[wi];
  const int n = w.n;
  if (P.budget_ctr) {
    advance_budget<T, false>(W[wi], P, sweep0, sigma, seed, sh);
    return;
  }
  for (int s = 0; s < n_sweeps; ++s)
    for (int k = 0; k < (P.step_limit > 0 ? min(n, P.step_limit) : n); ++k) {
      const long long idx = (long long)n_sweeps * w.log_base + (long long)s * n + k;
      mc_step<T>(w, P, k, seed, (uint32_t)(sweep0 + s), sigma, acc_log ? acc_log + idx : nullptr,
                 ratio_log ? ratio_log + idx : nullptr, sh);
    }
  if (threadIdx.x == 0) w.ctl->pos_valid = 0;  // every walker is at particle 0 of the next sweep
}

// Persistent sweeps with background refactorisation: a cluster of two CTAs per walker,
// rank 0 steps (as k_sweep), rank 1 factors (af_factor_loop).  launch_id: unique per
// launch of this context, > 0.
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_sweep_pair(const Walker* __restrict__ W, int walker0, Params P,
                                                     int n_sweeps, long long sweep0, double sigma,
                                                     const uint64_t* __restrict__ seeds, uint8_t* acc_log,
                                                     double* ratio_log, int launch_id) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const int wi = walker0 + (int)(blockIdx.x >> 1);
  const Walker& w0 = W[wi];
  if (blockIdx.x & 1) {
    af_factor_loop<T>(w0, P, launch_id, sh);
    return;
  }
  const uint64_t seed = seeds[wi];
  const int n = w0.n;
  if (P.budget_ctr) {
    advance_budget<T, true>(w0, P, sweep0, sigma, seed, sh);
  } else {
    for (int s = 0; s < n_sweeps; ++s)
      for (int k = 0; k < (P.step_limit > 0 ? min(n, P.step_limit) : n); ++k) {
        af_step_begin<T>(w0, P, sh);
        const Walker& w = active_of(w0);
        const long long idx = (long long)n_sweeps * w.log_base + (long long)s * n + k;
        mc_step<T>(w, P, k, seed, (uint32_t)(sweep0 + s), sigma, acc_log ? acc_log + idx : nullptr,
                   ratio_log ? ratio_log + idx : nullptr, sh);
      }
    if (threadIdx.x == 0) w0.ctl->pos_valid = 0;
  }
  if (threadIdx.x == 0) af_finish(w0, launch_id);
}

// One step (particle q of sweep s_local of a batch of n_sweeps) for every walker in the grid.
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_step(const Walker* __restrict__ W, int walker0, Params P, int q, int n_sweeps,
                                               int s_local, long long sweep0, double sigma,
                                               const uint64_t* __restrict__ seeds, uint8_t* acc_log, double* ratio_log,
                                               const long long* __restrict__ sweep_dev) {
  __shared__ Shared sh;
  const int wi = walker0 + blockIdx.x;
  const Walker& w = active_of(W[wi]);
  if (q >= w.n) return;
  ring_init(sh, P);
  if (sweep_dev) sweep0 = *sweep_dev;  // graph replays: the sweep index lives on the device
  const long long idx = (long long)n_sweeps * w.log_base + (long long)s_local * w.n + q;
  mc_step<T>(w, P, q, seeds[wi], (uint32_t)(sweep0 + s_local), sigma, acc_log ? acc_log + idx : nullptr,
             ratio_log ? ratio_log + idx : nullptr, sh);
}

// Single-move API: ratio for particle k moved to r_new (no commit); result in ctl.
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_ratio(const Walker* __restrict__ W, int wi, Params P, int k, double rx,
                                                double ry, double rz, int want_grad) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const Walker& w = active_of(W[wi]);
  Ctl* c = w.ctl;
  if (threadIdx.x == 0) {
    sh.rnew[0] = wrap_box(rx, w.L);
    sh.rnew[1] = wrap_box(ry, w.L);
    sh.rnew[2] = wrap_box(rz, w.L);
    c->pend_valid = 0;
  }
  __syncthreads();
  if (!build_move(w, k, sh)) return;
  SolveOut o;
  solve_with_controller<T>(w, P, k, o, sh);
  if (want_grad) {
    // column k of A'^{-1} is z / ratio (z = A^{-1} e_k, in x64), so at r':
    // grad ln|det A'| = sum_o grad phi_o(r') z_o / ratio with grad phi = -2 kappa (r' - Z_o) phi,
    // lap det A' / det A' = sum_o (4 kappa^2 d^2 - 6 kappa) phi z_o / ratio
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < sh.alen; t += blockDim.x) {
      const int col = sh.acol[t];
      const double* zo = w.Z + 3 * w.orb_of_col[col];
      const double dx = min_image(__dsub_rn(sh.rnew[0], zo[0]), w.L);
      const double dy = min_image(__dsub_rn(sh.rnew[1], zo[1]), w.L);
      const double dz = min_image(__dsub_rn(sh.rnew[2], zo[2]), w.L);
      const double pz = sh.aval[t] * w.x64[col];
      g[0] += -2.0 * w.kappa * dx * pz;
      g[1] += -2.0 * w.kappa * dy * pz;
      g[2] += -2.0 * w.kappa * dz * pz;
      g[3] += (4.0 * w.kappa * w.kappa * (dx * dx + dy * dy + dz * dz) - 6.0 * w.kappa) * pz;
    }
    for (int d = 0; d < 4; ++d) g[d] = block_sum(g[d], sh);
    if (threadIdx.x == 0) {
      for (int d = 0; d < 3; ++d) c->pend_grad[d] = g[d] / o.ratio;
      c->pend_lap = g[3] / o.ratio;
    }
  }
  for (int t = threadIdx.x; t < sh.alen; t += blockDim.x) { w.pend_acol[t] = sh.acol[t]; w.pend_aval[t] = sh.aval[t]; }
  for (int t = threadIdx.x; t < sh.ulen; t += blockDim.x) { w.pend_ucol[t] = sh.ucol[t]; w.pend_uval[t] = sh.uval[t]; }
  if (threadIdx.x == 0) {
    c->pend_alen = sh.alen;
    c->pend_ulen = sh.ulen;
    c->pend_k = k;
    c->pend_r[0] = sh.rnew[0]; c->pend_r[1] = sh.rnew[1]; c->pend_r[2] = sh.rnew[2];
    c->pend_ratio = o.ratio;
    c->pend_valid = o.status == ST_OK ? 1 : 0;
    c->proposals += 1;
  }
}

template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_accept(const Walker* __restrict__ W, int wi, Params P) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const Walker& w = active_of(W[wi]);
  Ctl* c = w.ctl;
  const int valid = c->pend_valid;
  const int k = c->pend_k;
  if (!valid) return;
  if (threadIdx.x == 0) {
    sh.alen = c->pend_alen; sh.ulen = c->pend_ulen;
    sh.rnew[0] = c->pend_r[0]; sh.rnew[1] = c->pend_r[1]; sh.rnew[2] = c->pend_r[2];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < sh.alen; t += blockDim.x) { sh.acol[t] = w.pend_acol[t]; sh.aval[t] = w.pend_aval[t]; }
  for (int t = threadIdx.x; t < sh.ulen; t += blockDim.x) { sh.ucol[t] = w.pend_ucol[t]; sh.uval[t] = w.pend_uval[t]; }
  __syncthreads();
  commit_move<T>(w, P, k, c->pend_ratio, sh);
  if (threadIdx.x == 0) { c->pend_valid = 0; c->accepts += 1; }
}

// Kinetic energy (Sec. 4 Eq. 21, read as (1/2n) sum_{p,o} (6 kappa - 4 kappa^2 |r_p - Z_o|^2)
// A_po (A^{-1})_op).  For every particle p the solve of a ratio, A z = e_p (z = column p
// of A^{-1}, indexed by orbital), contracted with the particle's own Slater row weighted by
// the Laplacian factor of each Gaussian; the weighted row takes the place of u, so the FP64
// refinement controls the error of this contraction.  One CTA per walker; out[walker].
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_kinetic(const Walker* __restrict__ W, Params P, double* out) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const Walker& w = active_of(W[blockIdx.x]);
  const int n = w.n, cap = w.cap;
  const double kap = w.kappa;
  double e = 0.0;
  for (int k = 0; k < n; ++k) {
    if (w.ctl->status != ST_OK) break;  // read by every thread after the last barrier
    const int len = w.a_len[k];
    const double rk[3] = {w.R[3 * k], w.R[3 * k + 1], w.R[3 * k + 2]};
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
      const int col = w.a_col[(size_t)k * cap + t];
      const double d2 = dist2(rk, w.Z + 3 * w.orb_of_col[col], w.L);
      sh.ucol[t] = col;
      sh.uval[t] = (6.0 * kap - 4.0 * kap * kap * d2) * w.a_val[(size_t)k * cap + t];
    }
    if (threadIdx.x == 0) sh.ulen = len;
    __syncthreads();
    SolveOut o;
    solve_with_controller<T>(w, P, k, o, sh);
    if (threadIdx.x == 0) e += o.ratio - 1.0;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = e / (2.0 * n);
}

// All Slater rows from the positions (warp per particle), then the initial pairing
// (particle i with orbital i), the greedy reordering and the first factorisation.
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_setup(const Walker* __restrict__ W, int walker0, Params P) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const Walker& w = active_of(W[walker0 + blockIdx.x]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Ctl* c = w.ctl;
  int bad = 0;
  for (int p = wid; p < w.n; p += nw) {
    const int len = build_row_warp(w, w.R + 3 * p, w.a_col + (size_t)p * w.cap, w.a_val + (size_t)p * w.cap, w.cap);
    if (lane == 0) {
      if (len < 0) bad = 1;
      w.a_len[p] = len < 0 ? 0 : len;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < w.n * w.cap; idx += blockDim.x) w.a_val32[idx] = (float)w.a_val[idx];
  for (int col = threadIdx.x; col < w.n; col += blockDim.x) {
    const int o = w.orb_of_col[col];
    w.part_of_row[col] = o;
    w.row_of_part[o] = col;
  }
  if (threadIdx.x == 0) {
    c->n_upd = 0;
    c->pend_valid = 0;
    c->its_sum = 0.0;
    c->its_cnt = 0;
  }
  __syncthreads();
  const int fl = factor_block<T>(w, P, sh, true);
  if (lane == 0 && bad) c->status = ST_CAPACITY;
  if (threadIdx.x == 0 && (fl & 2)) c->status = ST_CAPACITY;
}

template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_refactor(const Walker* __restrict__ W, int wi, Params P, int reorder) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const Walker& w = active_of(W[wi]);
  factor_block<T>(w, P, sh, reorder != 0);
}

// z = M v for the test entry point: v in r64 (FP64), result in x64 (FP64).
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_apply_precond(const Walker* __restrict__ W, int wi, Params P) {
  __shared__ Shared sh;
  const Walker& w = active_of(W[wi]);
  ring_init(sh, P);
  T* V = (T*)w.V;
  T* Zk = (T*)w.Zk;
  for (int i = threadIdx.x; i < w.n; i += blockDim.x) V[i] = (T)w.r64[i];
  __syncthreads();
  precond_apply<T>(w, P, V, Zk, sh);
  for (int i = threadIdx.x; i < w.n; i += blockDim.x) w.x64[i] = (double)Zk[i];
}

// Microbenchmark: `reps` back-to-back applications of one hot-path kernel per walker
// (0: L and U triangular solves, 1: SpMV in the working precision, 2: the full
// preconditioner apply with the update chain), on V[0] = 1 / sqrt(n).
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 2) k_bench(const Walker* __restrict__ W, Params P, int which, int reps) {
  __shared__ Shared sh;
  ring_init(sh, P);
  const Walker& w = active_of(W[blockIdx.x]);
  const int n = w.n;
  T* V = (T*)w.V;
  T* Zk = (T*)w.Zk;
  for (int i = threadIdx.x; i < n; i += blockDim.x) V[i] = (T)rsqrt((double)n);
  __syncthreads();
  for (int it = 0; it < reps; ++it) {
    if (which == 0) {
      const long long t0 = clock64();
      const T* y = tri_both<T>(w, P, V, sh);
      if (threadIdx.x == 0) w.ctl->cyc[PH_TRI] += clock64() - t0;
      block_scatter(Zk, w.perm, y, n);
      if (threadIdx.x == 0)
        w.ctl->alg_bytes += w.ctl->nnz_LU * (sizeof(T) + 4) + (double)n * (3 * sizeof(T) + 8);
    } else if (which == 1) {
      spmv<T>(w, P, stage_x<T>(w, P, V), Zk);
      if (threadIdx.x == 0) w.ctl->alg_bytes += w.ctl->nnz_A * (sizeof(T) + 4) + (double)n * (2 * sizeof(T) + 4);
    } else {
      precond_apply<T>(w, P, V, Zk, sh);
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// templated host launchers (one instantiation per working precision)
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t prep(K kernel, const LaunchCfg& L) {
  if (L.smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  return cudaSuccess;
}
#define VMC_LAUNCH(KERNEL, GRID, ...)                                   \
  do {                                                                 \
    cudaError_t e_ = prep(KERNEL, L);                                  \
    if (e_ != cudaSuccess) return e_;                                  \
    KERNEL<<<(GRID), L.threads, L.smem, L.stream>>>(__VA_ARGS__);      \
    return cudaGetLastError();                                         \
  } while (0)

template <typename T>
int kernel_static_smem_T() {
  cudaFuncAttributes a{};
  cudaFuncGetAttributes(&a, k_sweep<T>);
  return (int)a.sharedSizeBytes;
}
template <typename T>
cudaError_t launch_sweep_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int n_sweeps,
                           long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc, double* ratio) {
  VMC_LAUNCH(k_sweep<T>, nwalk, W, walker0, P, n_sweeps, sweep0, sigma, seeds, acc, ratio);
}
template <typename T>
cudaError_t launch_sweep_pair_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P,
                                int n_sweeps, long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc,
                                double* ratio, int launch_id) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(2 * nwalk);
  lc.blockDim = dim3(L.threads);
  lc.dynamicSmemBytes = L.smem;
  lc.stream = L.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = prep(k_sweep_pair<T>, L);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&lc, k_sweep_pair<T>, W, walker0, P, n_sweeps, sweep0, sigma, seeds, acc, ratio, launch_id);
}
template <typename T>
cudaError_t prepare_step_kernels_T(const LaunchCfg& L) { return prep(k_step<T>, L); }
template <typename T>
cudaError_t launch_step_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int q,
                          int n_sweeps, int s_local, long long sweep0, double sigma, const uint64_t* seeds,
                          uint8_t* acc, double* ratio, const long long* sweep_dev) {
  VMC_LAUNCH(k_step<T>, nwalk, W, walker0, P, q, n_sweeps, s_local, sweep0, sigma, seeds, acc, ratio, sweep_dev);
}
template <typename T>
cudaError_t launch_ratio_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int k, const double r[3],
                           int want_grad) {
  VMC_LAUNCH(k_ratio<T>, 1, W, wi, P, k, r[0], r[1], r[2], want_grad);
}
template <typename T>
cudaError_t launch_kinetic_T(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, double* out) {
  VMC_LAUNCH(k_kinetic<T>, nwalk, W, P, out);
}
template <typename T>
cudaError_t launch_accept_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P) {
  VMC_LAUNCH(k_accept<T>, 1, W, wi, P);
}
template <typename T>
cudaError_t launch_setup_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P) {
  VMC_LAUNCH(k_setup<T>, nwalk, W, walker0, P);
}
template <typename T>
cudaError_t launch_refactor_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int reorder) {
  VMC_LAUNCH(k_refactor<T>, 1, W, wi, P, reorder);
}
template <typename T>
cudaError_t launch_apply_precond_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P) {
  VMC_LAUNCH(k_apply_precond<T>, 1, W, wi, P);
}
template <typename T>
cudaError_t launch_bench_T(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, int which, int reps) {
  VMC_LAUNCH(k_bench<T>, nwalk, W, P, which, reps);
}

}  // namespace vmc
