// vmc_precond.cuh -- preconditioner construction on the device:
//   * the geometric particle/orbital reordering of Sec. 3.1 (greedy rule),
//   * ILUTP (Saad 1994; the threshold/pivoting variant the paper uses in Sec. 4):
//     row-wise IKJ elimination of A_p with dropping |w_j| < tau ||a_i||_2, at most
//     nl(i)+p entries kept in the L part and nu(i)+p in the U part, and a column
//     swap when permtol |w_j| > |w_i| for the largest U-part entry w_j (Sec. 3.2
//     Eq. 14: A Q ~ L U);
//   * level sets of L and U for the parallel triangular solves.
#pragma once
#include "vmc_geom.cuh"

namespace vmc {

// ---------------------------------------------------------------------------
// Greedy reordering (Sec. 3.1): for i = 0..n-2, find the orbital nearest to the
// particle at position i among positions >= i and swap it into column i; if the
// nearest is already at i, find the particle nearest to orbital i among positions
// >= i and swap it into row i.  Ties go to the lowest position.  Positions are the
// current columns; afterwards orbitals return to their fixed columns carrying their
// new partner particle, so only part_of_row / row_of_part change.
// Block-wide; O(n^2) distance evaluations.
// ---------------------------------------------------------------------------
__device__ __noinline__ void reorder_block(const Walker& w, Shared& sh) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x;
  for (int c = tid; c < n; c += nt) { w.gP[c] = w.part_of_row[c]; w.gQ[c] = w.orb_of_col[c]; }
  __syncthreads();
  for (int i = 0; i < n - 1; ++i) {
    const int p = w.gP[i];
    const double rp[3] = {w.R[3 * p], w.R[3 * p + 1], w.R[3 * p + 2]};
    double bd = 1e300;
    int bj = 0x7fffffff;
    for (int j = i + tid; j < n; j += nt) {
      const double d = dist2(rp, w.Z + 3 * w.gQ[j], w.L);
      if (d < bd) { bd = d; bj = j; }
    }
    block_argmin(bd, bj, sh);
    if (bj != i) {
      if (tid == 0) { const int t = w.gQ[i]; w.gQ[i] = w.gQ[bj]; w.gQ[bj] = t; }
    } else {
      const int o = w.gQ[i];
      const double* zo = w.Z + 3 * o;
      double bd2 = 1e300;
      int bk = 0x7fffffff;
      for (int k = i + tid; k < n; k += nt) {
        const int q = w.gP[k];
        const double d = dist2(w.R + 3 * q, zo, w.L);
        if (d < bd2) { bd2 = d; bk = k; }
      }
      block_argmin(bd2, bk, sh);
      if (bk != i && tid == 0) { const int t = w.gP[i]; w.gP[i] = w.gP[bk]; w.gP[bk] = t; }
    }
    __syncthreads();
  }
  for (int g = tid; g < n; g += nt) {
    const int c = w.col_of_orb[w.gQ[g]];
    const int p = w.gP[g];
    w.part_of_row[c] = p;
    w.row_of_part[p] = c;
  }
  __syncthreads();
}

// Rank-based top-k of the compacted candidates sh.selF/selV[0..c): keep[e] = rank < keep.
// Larger magnitude first, ties to the smaller label.
__device__ __forceinline__ bool sel_keep(const Shared& sh, int c, int e, int keep) {
  if (c <= keep) return true;
  const double me = fabs(sh.selV[e]);
  const int fe = sh.selF[e];
  int rank = 0;
  for (int o = 0; o < c; ++o) {
    const double mo = fabs(sh.selV[o]);
    rank += (mo > me) || (mo == me && sh.selF[o] < fe);
  }
  return rank < keep;
}

// ---------------------------------------------------------------------------
// ILUTP, performed by warp 0 of the CTA (rows are sequential); the caller
// synchronises the block afterwards.  U rows are stored with ORIGINAL column
// labels while the factorisation runs (later pivots relabel columns >= i only)
// and relabelled to factor labels by relabel_and_levels().
// Returns: bit 0 breakdown (zero pivot replaced by (1e-4 + tau) ||a_i||), bit 1
// capacity overflow.
// ---------------------------------------------------------------------------
__device__ __noinline__ int ilutp_warp(const Walker& w, const Params& P, Shared& sh, int* npiv_out, double* nnz_out,
                          int* p_out) {
  const int n = w.n, lane = threadIdx.x & 31, cap = w.cap, capLU = w.capLU;
  int p = P.lfil_extra;
  if (p < 0) {
    long long tot = 0;
    for (int i = lane; i < n; i += 32) tot += w.a_len[i];
    tot = warp_sum_ll(tot);
    p = (int)((tot + 2LL * n - 1) / (2LL * n));  // ceil(avg nnz per row / 2)
  }
  p = min(p, (capLU - 2) / 2);
  const int pk = max(0, min(p, capLU - 2 - cap));  // never exceeds the row capacity
  for (int i = lane; i < n; i += 32) {
    w.perm[i] = i; w.iperm[i] = i; w.wpos[i] = -1; w.wrow[i] = 0.0; w.lev_l[i] = 0;
  }
  __syncwarp();
  int npiv = 0, flags = 0;
  double nnz = 0.0;
  for (int r = 0; r < n; ++r) {
    const int part = w.part_of_row[r];
    const int len = w.a_len[part];
    const int* ac = w.a_col + (size_t)part * cap;
    const double* av = w.a_val + (size_t)part * cap;
    double ss = 0.0;
    int nl = 0, nu = 0;
    for (int t = lane; t < len; t += 32) {
      const int f = w.iperm[ac[t]];
      const double v = av[t];
      w.wrow[f] = v;
      w.wpos[f] = t;
      sh.nz[t] = f;
      ss += v * v;
      nl += f < r;
      nu += f > r;
    }
    ss = warp_sum(ss);
    nl = warp_sum_int(nl);
    nu = warp_sum_int(nu);
    int cnt = len;
    const double norm = sqrt(ss);
    const double thr = P.drop_tol * norm;
    __syncwarp();
    // --- elimination with the previous U rows, in increasing label order ---
    int last = -1;
    for (;;) {
      int best = 0x7fffffff;
      for (int t = lane; t < cnt; t += 32) {
        const int f = sh.nz[t];
        if (f > last && f < r && f < best) best = f;
      }
      best = warp_min_int(best);
      if (best == 0x7fffffff) break;
      last = best;
      const double wk = w.wrow[best] * w.u_dinv64[best];
      __syncwarp();
      if (fabs(wk) < thr) {
        if (lane == 0) w.wrow[best] = 0.0;  // dropped multiplier
        __syncwarp();
        continue;
      }
      if (lane == 0) w.wrow[best] = wk;
      const int ul = w.u_len[best];
      const int* uc = w.u_col + (size_t)best * capLU;
      const double* uv = w.u_val64 + (size_t)best * capLU;
      for (int base = 0; base < ul; base += 32) {
        const int t = base + lane;
        const bool valid = t < ul;
        int f = 0;
        double v = 0.0;
        bool exists = false;
        if (valid) { f = w.iperm[uc[t]]; v = uv[t]; exists = w.wpos[f] >= 0; }
        const unsigned nm = __ballot_sync(0xffffffffu, valid && !exists);
        const int slot = cnt + __popc(nm & lanemask_lt());
        if (valid) {
          if (!exists) {
            if (slot < kMaxRowNZ) { sh.nz[slot] = f; w.wpos[f] = slot; w.wrow[f] = -wk * v; }
          } else {
            w.wrow[f] -= wk * v;
          }
        }
        cnt += __popc(nm);
        __syncwarp();
      }
      if (cnt > kMaxRowNZ) { flags |= 2; cnt = kMaxRowNZ; }
    }
    // --- L part: keep the nl + p largest multipliers ---
    int cL = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int t = base + lane;
      bool c = false;
      int f = 0;
      double v = 0.0;
      if (t < cnt) { f = sh.nz[t]; v = w.wrow[f]; c = f < r && v != 0.0; }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      const int slot = cL + __popc(m & lanemask_lt());
      if (c && slot < kMaxSel) { sh.selF[slot] = f; sh.selV[slot] = v; }
      cL += __popc(m);
    }
    if (cL > kMaxSel) { flags |= 2; cL = kMaxSel; }
    __syncwarp();
    const int keepL = nl + pk;
    int nL = 0, levmax = -1;
    for (int base = 0; base < cL; base += 32) {
      const int e = base + lane;
      const bool k = e < cL && sel_keep(sh, cL, e, keepL);
      const unsigned m = __ballot_sync(0xffffffffu, k);
      const int slot = nL + __popc(m & lanemask_lt());
      if (k && slot < capLU) {
        w.l_col[(size_t)r * capLU + slot] = sh.selF[e];
        w.l_val64[(size_t)r * capLU + slot] = sh.selV[e];
        levmax = max(levmax, w.lev_l[sh.selF[e]]);
      }
      nL += __popc(m);
    }
    levmax = warp_max_int(levmax);
    if (nL > capLU) { flags |= 2; nL = capLU; }
    __syncwarp();
    // --- U part: entries above threshold, keep the nu + p largest ---
    double dval = w.wpos[r] >= 0 ? w.wrow[r] : 0.0;
    int cU = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int t = base + lane;
      bool c = false;
      int f = 0;
      double v = 0.0;
      if (t < cnt) { f = sh.nz[t]; v = w.wrow[f]; c = f > r && fabs(v) >= thr && v != 0.0; }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      const int slot = cU + __popc(m & lanemask_lt());
      if (c && slot < kMaxSel) { sh.selF[slot] = f; sh.selV[slot] = v; }
      cU += __popc(m);
    }
    if (cU > kMaxSel) { flags |= 2; cU = kMaxSel; }
    __syncwarp();
    const int keepU = nu + pk;
    // mark kept entries by negating the label (-f-1); compact afterwards
    bool mykeep[kMaxSel / 32];
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      mykeep[q] = e < cU && sel_keep(sh, cU, e, keepU);
    }
    __syncwarp();
    // pivot: the largest kept U entry (ties: smaller label)
    double bv = 0.0;
    int bf = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      if (mykeep[q]) {
        const double v = fabs(sh.selV[e]);
        const int f = sh.selF[e];
        if (v > bv || (v == bv && f < bf)) { bv = v; bf = f; }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int f2 = __shfl_xor_sync(0xffffffffu, bf, o);
      if (v2 > bv || (v2 == bv && f2 < bf)) { bv = v2; bf = f2; }
    }
    int jm = -1;
    if (bf != 0x7fffffff && P.permtol * bv > fabs(dval)) jm = bf;
    double newdiag = dval;
    if (jm >= 0) {
      // the column labelled jm becomes the diagonal; the old diagonal value moves
      // to label jm (a U-part entry, or nothing if it was zero)
      newdiag = w.wrow[jm];
      if (lane == 0) {
        const int cr = w.perm[r], cj = w.perm[jm];
        w.perm[r] = cj; w.perm[jm] = cr;
        w.iperm[cj] = r; w.iperm[cr] = jm;
      }
      ++npiv;
    }
    __syncwarp();
    int nU = 0;
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      bool k = mykeep[q];
      double v = 0.0;
      int f = 0;
      if (k) {
        f = sh.selF[e];
        v = sh.selV[e];
        if (f == jm) { v = dval; k = dval != 0.0; }
      }
      const unsigned m = __ballot_sync(0xffffffffu, k);
      const int slot = nU + __popc(m & lanemask_lt());
      if (k && slot < capLU) {
        w.u_col[(size_t)r * capLU + slot] = w.perm[f];  // original column label
        w.u_val64[(size_t)r * capLU + slot] = v;
      }
      nU += __popc(m);
    }
    if (nU > capLU) { flags |= 2; nU = capLU; }
    if (newdiag == 0.0) {
      newdiag = (1e-4 + P.drop_tol) * (norm > 0.0 ? norm : 1.0);
      flags |= 1;
    }
    if (lane == 0) {
      w.l_len[r] = nL;
      w.u_len[r] = nU;
      w.u_dinv64[r] = 1.0 / newdiag;
      w.lev_l[r] = levmax + 1;
    }
    nnz += (double)(nL + nU + 1);
    // clear the working row
    for (int t = lane; t < cnt; t += 32) {
      const int f = sh.nz[t];
      w.wpos[f] = -1;
      w.wrow[f] = 0.0;
    }
    __syncwarp();
  }
  *npiv_out = npiv;
  *nnz_out = nnz;
  *p_out = p;
  return flags;
}

// Block-wide: relabel U columns to factor labels, compute U levels (warp 0,
// reverse order) and pack both level sets (counting sort by level).
template <typename T>
__device__ __noinline__ void relabel_and_levels(const Walker& w, Shared& sh) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x, capLU = w.capLU;
  for (int idx = tid; idx < n * capLU; idx += nt) {
    const int r = idx / capLU, t = idx - r * capLU;
    if (t < w.u_len[r]) w.u_col[idx] = w.iperm[w.u_col[idx]];
  }
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    for (int r = n - 1; r >= 0; --r) {
      const int ul = w.u_len[r];
      int lv = -1;
      for (int t = lane; t < ul; t += 32) lv = max(lv, w.lev_u[w.u_col[(size_t)r * capLU + t]]);
      lv = warp_max_int(lv);
      if (lane == 0) w.lev_u[r] = lv + 1;
      __syncwarp();
    }
  }
  __syncthreads();
  // level counts
  int mlv = 0, muv = 0;
  for (int r = tid; r < n; r += nt) { mlv = max(mlv, w.lev_l[r]); muv = max(muv, w.lev_u[r]); }
  const int ml = block_max_int(mlv, sh);
  const int mu = block_max_int(muv, sh);
  const int nll = ml + 1, nlu = mu + 1;
  for (int q = tid; q <= n; q += nt) { w.l_lvl_ptr[q] = 0; w.u_lvl_ptr[q] = 0; }
  __syncthreads();
  for (int r = tid; r < n; r += nt) {
    atomicAdd(&w.l_lvl_ptr[w.lev_l[r] + 1], 1);
    atomicAdd(&w.u_lvl_ptr[w.lev_u[r] + 1], 1);
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < nll; ++q) w.l_lvl_ptr[q + 1] += w.l_lvl_ptr[q];
    for (int q = 0; q < nlu; ++q) w.u_lvl_ptr[q + 1] += w.u_lvl_ptr[q];
  }
  __syncthreads();
  for (int q = tid; q < nll; q += nt) w.lvl_cur[q] = w.l_lvl_ptr[q];
  __syncthreads();
  for (int r = tid; r < n; r += nt) w.l_lvl_rows[atomicAdd(&w.lvl_cur[w.lev_l[r]], 1)] = r;
  __syncthreads();
  for (int q = tid; q < nlu; q += nt) w.lvl_cur[q] = w.u_lvl_ptr[q];
  __syncthreads();
  for (int r = tid; r < n; r += nt) w.u_lvl_rows[atomicAdd(&w.lvl_cur[w.lev_u[r]], 1)] = r;
  // working-precision copies of the factors
  if (sizeof(T) != sizeof(double)) {
    T* lv = (T*)w.l_valT;
    T* uv = (T*)w.u_valT;
    T* dv = (T*)w.u_dinvT;
    for (int idx = tid; idx < n * capLU; idx += nt) {
      lv[idx] = (T)w.l_val64[idx];
      uv[idx] = (T)w.u_val64[idx];
    }
    for (int r = tid; r < n; r += nt) dv[r] = (T)w.u_dinv64[r];
  }
  if (tid == 0) { w.ctl->nlev_l = nll; w.ctl->nlev_u = nlu; }
  __syncthreads();
}

// Full (re)factorisation: optional reorder, ILUTP, levels; clears the update chain.
// Block-wide.  Returns the ILUTP flags.
template <typename T>
__device__ __noinline__ int factor_block(const Walker& w, const Params& P, Shared& sh, bool reorder) {
  if (reorder) reorder_block(w, sh);
  if (threadIdx.x < 32) {
    int npiv = 0, p = 0;
    double nnz = 0.0;
    for (int r = threadIdx.x; r < w.n; r += 32) w.lev_u[r] = 0;
    const int fl = ilutp_warp(w, P, sh, &npiv, &nnz, &p);
    if (threadIdx.x == 0) {
      sh.iflag[0] = fl;
      Ctl* c = w.ctl;
      c->last_pivots = npiv;
      c->nnz_LU = nnz;
      c->p_lfil = p;
      c->factorizations += 1;
      c->n_upd = 0;
      c->last_breakdown = fl & 1;
    }
  }
  __syncthreads();
  const int fl = sh.iflag[0];
  relabel_and_levels<T>(w, sh);
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int i = 0; i < w.n; ++i) tot += w.a_len[i];
    w.ctl->nnz_A = (double)tot;
  }
  __syncthreads();
  return fl;
}

}  // namespace vmc
