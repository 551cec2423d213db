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
static __device__ __noinline__ void reorder_block(const Walker& w, Shared& sh) {
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

// Top-k of the compacted candidates sh.selF/selV[0..c) by magnitude (ties: smaller
// label), by one warp: a histogram of binary exponents below the largest one (bins
// of one octave, the last bin collecting everything smaller) finds the octave that
// holds the k-th largest; entries in higher octaves are kept, entries in that octave
// are ranked among themselves.  Result in sh.selK[0..c).
template <typename W>
__device__ __forceinline__ int octave_bin(W v, int emax) {
  int e;
  frexp(v, &e);
  return min(63, max(0, emax - e));
}
template <typename W>
__device__ void select_topk(Shared& sh, int c, int keep) {
  const int lane = threadIdx.x & 31;
  const W* sv = reinterpret_cast<const W*>(sh.selV);
  if (c <= keep) {
    for (int e = lane; e < c; e += 32) sh.selK[e] = 1;
    __syncwarp();
    return;
  }
  W vmax = 0;
  for (int e = lane; e < c; e += 32) vmax = fmax(vmax, fabs(sv[e]));
#pragma unroll
  for (int o = 16; o; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  int emax;
  frexp(vmax, &emax);
  for (int b = lane; b < 64; b += 32) sh.hist[b] = 0;
  __syncwarp();
  for (int e = lane; e < c; e += 32) atomicAdd(&sh.hist[octave_bin<W>(fabs(sv[e]), emax)], 1);
  __syncwarp();
  // boundary bin bb: count(bins < bb) < keep <= count(bins <= bb)
  int h0 = sh.hist[lane], h1 = sh.hist[lane + 32];
  int inc0 = h0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) { const int v = __shfl_up_sync(0xffffffffu, inc0, o); if (lane >= o) inc0 += v; }
  const int tot0 = __shfl_sync(0xffffffffu, inc0, 31);
  int inc1 = h1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) { const int v = __shfl_up_sync(0xffffffffu, inc1, o); if (lane >= o) inc1 += v; }
  inc1 += tot0;
  const unsigned m0 = __ballot_sync(0xffffffffu, inc0 >= keep);
  const unsigned m1 = __ballot_sync(0xffffffffu, inc1 >= keep);
  const int bb = m0 ? __ffs(m0) - 1 : 32 + __ffs(m1) - 1;
  const int below = (bb < 32 ? __shfl_sync(0xffffffffu, inc0 - h0, bb & 31)
                             : __shfl_sync(0xffffffffu, inc1 - h1, bb & 31));
  const int need = keep - below;  // entries to keep from the boundary bin
  // compact the boundary octave, decide the others
  int cb = 0;
  for (int base = 0; base < c; base += 32) {
    const int e = base + lane;
    int b = 64;
    if (e < c) {
      b = octave_bin<W>(fabs(sv[e]), emax);
      sh.selK[e] = b < bb ? 1 : 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, b == bb);
    const int slot = cb + __popc(m & lanemask_lt());
    if (b == bb && slot < 256) sh.bndE[slot] = e;
    cb += __popc(m);
  }
  __syncwarp();
  if (cb <= 256) {
    for (int q = lane; q < cb; q += 32) {
      const int e = sh.bndE[q];
      const W me = fabs(sv[e]);
      const int fe = sh.selF[e];
      int rank = 0;
      for (int o = 0; o < cb; ++o) {
        const int eo = sh.bndE[o];
        const W mo = fabs(sv[eo]);
        rank += (mo > me) || (mo == me && sh.selF[eo] < fe);
      }
      sh.selK[e] = rank < need ? 1 : 0;
    }
  } else {
    for (int e = lane; e < c; e += 32) {
      const W me = fabs(sv[e]);
      if (octave_bin<W>(me, emax) != bb) continue;
      const int fe = sh.selF[e];
      int rank = 0;
      for (int o = 0; o < c; ++o) {
        const W mo = fabs(sv[o]);
        if (octave_bin<W>(mo, emax) != bb) continue;
        rank += (mo > me) || (mo == me && sh.selF[o] < fe);
      }
      sh.selK[e] = rank < need ? 1 : 0;
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// ILUTP, performed by warp 0 of the CTA (rows are sequential); the caller
// synchronises the block afterwards.  The working row, multipliers, drop and pivot
// tests run in the engine's working precision T (FP64 engine: FP64; mixed engine:
// FP32, the precision its factors are stored and applied in -- a warp-serial FP64
// elimination step costs ~1000 cycles on GB300, whose FP64 rate is 1/48 of FP32);
// row norms are accumulated in FP64.  U rows are stored with ORIGINAL column
// labels while the factorisation runs (later pivots relabel columns >= i only)
// and relabelled to factor labels by relabel_and_levels().
// Returns: bit 0 breakdown (zero pivot replaced by (1e-4 + tau) ||a_i||), bit 1
// capacity overflow.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int ilutp_warp(const Walker& w, const Params& P, Shared& sh, int* npiv_out, double* nnz_out,
                                       int* p_out) {
  const int n = w.n, lane = threadIdx.x & 31, cap = w.cap, capLU = w.capLU;
  // Working arrays in the dynamic shared memory (idle while factoring) when they fit:
  // wrow (dense work row), wpos (its slot map), iperm, then U diagonal inverses,
  // U lengths and L levels.  Otherwise the global copies are used.
  const size_t dbytes = (size_t)P.dsm_bytes;
  unsigned char* dsm = dyn_smem();
  T* wrow = reinterpret_cast<T*>(w.wrow);
  int* wpos = w.wpos;
  int* iperm = w.iperm;
  T* udinv = reinterpret_cast<T*>(w.u_dinv64);
  int* ulen_a = w.u_len;
  int* levl = w.lev_l;
  // Pending L-part labels of the current row: a bitmap over labels (one bit per
  // label) with a summary word per 32 bitmap words, so that the next label to
  // eliminate is found with two warp-wide word scans instead of a scan of the row.
  // They take n/8 bytes and come first, so they stay in shared memory at any n.
  const int nwords = (n + 31) >> 5;
  const int nsum = (nwords + 31) >> 5;
  unsigned* lbits = nullptr;
  unsigned* lsum = nullptr;
  const size_t bm_bytes = 4 * (size_t)(pad4(nwords) + pad4(nsum));
  size_t base = 0;
  if (bm_bytes <= dbytes) {
    lbits = (unsigned*)dsm;
    lsum = lbits + pad4(nwords);
    base = (bm_bytes + 15) & ~(size_t)15;
  }
  const bool sm_work = base + (size_t)16 * n <= dbytes;
  const bool sm_rows = base + (size_t)32 * n <= dbytes;
  if (sm_work) {
    wrow = (T*)(dsm + base);
    wpos = (int*)(dsm + base + (size_t)8 * n);
    iperm = wpos + n;
  }
  if (sm_rows) {
    udinv = (T*)(dsm + base + (size_t)16 * n);
    ulen_a = (int*)(dsm + base + (size_t)24 * n);
    levl = ulen_a + n;
  }
  // without shared memory the U diagonal lives in the global FP64 array as T values;
  // it is rewritten as FP64 inverses at the end
  // Cache of finished U rows (original labels; values in the working precision):
  // row r at ucc/ucv[uoff[r] .. uoff[r] + len), uoff[r] = -1 when not cached.
  int* uoff = nullptr;
  int* ucc = nullptr;
  T* ucv = nullptr;
  int ucap = 0, ufill = 0;
  const size_t cache_at = base + (size_t)32 * n;
  if (sm_rows && cache_at + (size_t)4 * n + 16 + 64 * (sizeof(T) + 4) <= dbytes) {
    uoff = (int*)(dsm + cache_at);
    const size_t rest = dbytes - cache_at - (size_t)4 * pad4(n + 1);
    ucap = (int)(rest / (sizeof(T) + 4)) & ~3;
    ucc = uoff + pad4(n + 1);
    ucv = (T*)(ucc + ucap);
  }
  if (lbits) {
    for (int i = lane; i < nwords; i += 32) lbits[i] = 0u;
    for (int i = lane; i < nsum; i += 32) lsum[i] = 0u;
  }
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
    w.perm[i] = i; iperm[i] = i; wpos[i] = -1; wrow[i] = (T)0; levl[i] = 0;
  }
  __syncwarp();
  int npiv = 0, flags = 0;
  long long n_elim = 0, n_cand = 0;
  double nnz = 0.0;
  for (int r = 0; r < n; ++r) {
    const int part = w.part_of_row[r];
    const int len = w.a_len[part];
    const int* ac = w.a_col + (size_t)part * cap;
    const double* av = w.a_val + (size_t)part * cap;
    double ss = 0.0;
    int nl = 0, nu = 0;
    for (int t = lane; t < len; t += 32) {
      const int f = iperm[ac[t]];
      const double v = av[t];
      wrow[f] = (T)v;
      wpos[f] = t;
      sh.nz[t] = f;
      ss += v * v;
      nl += f < r;
      nu += f > r;
      if (lbits && f < r) {
        atomicOr(&lbits[f >> 5], 1u << (f & 31));
        atomicOr(&lsum[f >> 10], 1u << ((f >> 5) & 31));
      }
    }
    ss = warp_sum(ss);
    nl = warp_sum_int(nl);
    nu = warp_sum_int(nu);
    int cnt = len;
    const double norm = sqrt(ss);
    const T thr = (T)(P.drop_tol * norm);
    __syncwarp();
    // --- elimination with the previous U rows, in increasing label order ---
    int last = -1;
    for (;;) {
      int best = 0x7fffffff;
      if (lbits) {
        __syncwarp();
        // next pending label > last: first the rest of last's word, then the summary
        const int w0 = (last + 1) >> 5;
        unsigned cur = w0 < nwords ? lbits[w0] & (0xffffffffu << ((last + 1) & 31)) : 0u;
        if (w0 < nwords && (last + 1) >= 0 && cur) {
          best = (w0 << 5) + __ffs(cur) - 1;
        } else {
          const int s0 = (w0 + 1) >> 5;  // summary word holding bitmap word w0 + 1
          for (int sb = s0; sb < nsum && best == 0x7fffffff; sb += 32) {
            const int si = sb + lane;
            unsigned sv = si < nsum ? lsum[si] : 0u;
            if (si == s0) sv &= 0xffffffffu << ((w0 + 1) & 31);
            const unsigned any = __ballot_sync(0xffffffffu, sv != 0u);
            if (any) {
              const int src = __ffs(any) - 1;
              const unsigned svs = __shfl_sync(0xffffffffu, sv, src);
              const int word = ((sb + src) << 5) + __ffs(svs) - 1;
              best = (word << 5) + __ffs(lbits[word]) - 1;
            }
          }
        }
        if (best >= r) best = 0x7fffffff;
      } else {
        for (int t = lane; t < cnt; t += 32) {
          const int f = sh.nz[t];
          if (f > last && f < r && f < best) best = f;
        }
        best = warp_min_int(best);
      }
      if (best == 0x7fffffff) break;
      last = best;
      ++n_elim;
      const T wk = wrow[best] * udinv[best];
      __syncwarp();
      if (fabs(wk) < thr) {
        if (lane == 0) wrow[best] = (T)0;  // dropped multiplier
        __syncwarp();
        continue;
      }
      if (lane == 0) wrow[best] = wk;
      const int ul = ulen_a[best];
      const int ub = uoff ? uoff[best] : -1;
      for (int base = 0; base < ul; base += 32) {
        const int t = base + lane;
        const bool valid = t < ul;
        int f = 0;
        T v = 0;
        bool exists = false;
        if (valid) {
          if (ub >= 0) { f = iperm[ucc[ub + t]]; v = ucv[ub + t]; }
          else { f = iperm[w.u_col[(size_t)best * capLU + t]]; v = (T)w.u_val64[(size_t)best * capLU + t]; }
          exists = wpos[f] >= 0;
        }
        const unsigned nm = __ballot_sync(0xffffffffu, valid && !exists);
        const int slot = cnt + __popc(nm & lanemask_lt());
        if (valid) {
          if (!exists) {
            if (slot < kMaxRowNZ) {
              sh.nz[slot] = f; wpos[f] = slot; wrow[f] = -wk * v;
              if (lbits && f < r) {
                atomicOr(&lbits[f >> 5], 1u << (f & 31));
                atomicOr(&lsum[f >> 10], 1u << ((f >> 5) & 31));
              }
            }
          } else {
            wrow[f] -= wk * v;
          }
        }
        cnt += __popc(nm);
        __syncwarp();
      }
      if (cnt > kMaxRowNZ) { flags |= 2; cnt = kMaxRowNZ; }
    }
    n_cand += cnt;
    // --- L part: keep the nl + p largest multipliers ---
    T* selv = reinterpret_cast<T*>(sh.selV);
    int cL = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int t = base + lane;
      bool c = false;
      int f = 0;
      T v = 0;
      if (t < cnt) { f = sh.nz[t]; v = wrow[f]; c = f < r && v != (T)0; }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      const int slot = cL + __popc(m & lanemask_lt());
      if (c && slot < kMaxSel) { sh.selF[slot] = f; selv[slot] = v; }
      cL += __popc(m);
    }
    if (cL > kMaxSel) { flags |= 2; cL = kMaxSel; }
    __syncwarp();
    const int keepL = nl + pk;
    select_topk<T>(sh, cL, keepL);
    int nL = 0, levmax = -1;
    for (int base = 0; base < cL; base += 32) {
      const int e = base + lane;
      const bool k = e < cL && sh.selK[e];
      const unsigned m = __ballot_sync(0xffffffffu, k);
      const int slot = nL + __popc(m & lanemask_lt());
      if (k && slot < capLU) {
        w.l_col[(size_t)r * capLU + slot] = sh.selF[e];
        w.l_val64[(size_t)r * capLU + slot] = (double)selv[e];
        levmax = max(levmax, levl[sh.selF[e]]);
      }
      nL += __popc(m);
    }
    levmax = warp_max_int(levmax);
    if (nL > capLU) { flags |= 2; nL = capLU; }
    __syncwarp();
    // --- U part: entries above threshold, keep the nu + p largest ---
    T dval = wpos[r] >= 0 ? wrow[r] : (T)0;
    int cU = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int t = base + lane;
      bool c = false;
      int f = 0;
      T v = 0;
      if (t < cnt) { f = sh.nz[t]; v = wrow[f]; c = f > r && fabs(v) >= thr && v != (T)0; }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      const int slot = cU + __popc(m & lanemask_lt());
      if (c && slot < kMaxSel) { sh.selF[slot] = f; selv[slot] = v; }
      cU += __popc(m);
    }
    if (cU > kMaxSel) { flags |= 2; cU = kMaxSel; }
    __syncwarp();
    const int keepU = nu + pk;
    select_topk<T>(sh, cU, keepU);
    bool mykeep[kMaxSel / 32];
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      mykeep[q] = e < cU && sh.selK[e];
    }
    __syncwarp();
    // pivot: the largest kept U entry (ties: smaller label)
    T bv = 0;
    int bf = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      if (mykeep[q]) {
        const T v = fabs(selv[e]);
        const int f = sh.selF[e];
        if (v > bv || (v == bv && f < bf)) { bv = v; bf = f; }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int f2 = __shfl_xor_sync(0xffffffffu, bf, o);
      if (v2 > bv || (v2 == bv && f2 < bf)) { bv = v2; bf = f2; }
    }
    int jm = -1;
    if (bf != 0x7fffffff && (T)P.permtol * bv > fabs(dval)) jm = bf;
    T newdiag = dval;
    if (jm >= 0) {
      // the column labelled jm becomes the diagonal; the old diagonal value moves
      // to label jm (a U-part entry, or nothing if it was zero)
      newdiag = wrow[jm];
      if (lane == 0) {
        const int cr = w.perm[r], cj = w.perm[jm];
        w.perm[r] = cj; w.perm[jm] = cr;
        iperm[cj] = r; iperm[cr] = jm;
      }
      ++npiv;
    }
    __syncwarp();
    int nU = 0;
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      bool k = mykeep[q];
      T v = 0;
      int f = 0;
      if (k) {
        f = sh.selF[e];
        v = selv[e];
        if (f == jm) { v = dval; k = dval != (T)0; }
      }
      const unsigned m = __ballot_sync(0xffffffffu, k);
      const int slot = nU + __popc(m & lanemask_lt());
      if (k && slot < capLU) {
        const int oc = w.perm[f];  // original column label
        w.u_col[(size_t)r * capLU + slot] = oc;
        w.u_val64[(size_t)r * capLU + slot] = (double)v;
        if (uoff && ufill + slot < ucap) { ucc[ufill + slot] = oc; ucv[ufill + slot] = v; }
      }
      nU += __popc(m);
    }
    if (nU > capLU) { flags |= 2; nU = capLU; }
    if (uoff) {
      if (lane == 0) uoff[r] = ufill + nU <= ucap ? ufill : -1;
      if (ufill + nU <= ucap) ufill += nU;
    }
    if (newdiag == 0.0) {
      newdiag = (1e-4 + P.drop_tol) * (norm > 0.0 ? norm : 1.0);
      flags |= 1;
    }
    if (lane == 0) {
      w.l_len[r] = nL;
      ulen_a[r] = nU;
      udinv[r] = 1.0 / newdiag;
      levl[r] = levmax + 1;
    }
    nnz += (double)(nL + nU + 1);
    // clear the working row (and the pending-label bitmaps)
    for (int t = lane; t < cnt; t += 32) {
      const int f = sh.nz[t];
      wpos[f] = -1;
      wrow[f] = (T)0;
      if (lbits && f < r) { lbits[f >> 5] = 0u; lsum[f >> 10] = 0u; }
    }
    __syncwarp();
  }
  __syncwarp();
  if (sm_work)
    for (int i = lane; i < n; i += 32) w.iperm[i] = iperm[i];
  if (sm_rows) {
    for (int i = lane; i < n; i += 32) { w.u_dinv64[i] = (double)udinv[i]; w.u_len[i] = ulen_a[i]; w.lev_l[i] = levl[i]; }
  } else if (sizeof(T) != sizeof(double)) {
    // udinv aliased the global FP64 array as T values: widen in place, back to front
    __syncwarp();
    if (lane == 0)
      for (int i = n - 1; i >= 0; --i) w.u_dinv64[i] = (double)udinv[i];
  }
  __syncwarp();
  if (lane == 0) { w.ctl->ilu_rows += n; w.ctl->ilu_elims += n_elim; w.ctl->ilu_cand += n_cand; }
  *npiv_out = npiv;
  *nnz_out = nnz;
  *p_out = p;
  return flags;
}

// ---------------------------------------------------------------------------
// ILUTP with the working row in shared memory (the same elimination, drop, lfil and
// pivot rules as ilutp_warp, in the same order, so the factors are the same).
//   * The working row is an open-addressing hash map keyed by factor label (linear
//     probing, a table of HS slots for at most HS/2 candidates): its entries' labels in
//     sh.nz[t], values in wv[t], hash slot in hslot[t].
//   * The inverse column permutation is held in shared memory as 16-bit labels
//     (n <= 65535).
//   * A U row is read with its header {1/u_rr, length} (u_head) in one round trip: the
//     lanes load the header and the row's first 64 slots together, before the length
//     is known.  When shared memory is left over (small n) the finished U rows, their
//     inverse diagonals and lengths are also cached there, as in ilutp_warp.
// One warp; the caller synchronises the block afterwards.  Returns the ilutp_warp flags.
// ---------------------------------------------------------------------------
struct IluSm {
  int ok, HS, lgHS, maxc, cache;
  unsigned o_bits, o_sum, o_ip, o_hkey, o_hidx, o_hslot, o_wv, o_meta, o_len, o_uoff, o_cc, ucap;
};
template <typename T>
__device__ __forceinline__ IluSm ilu_sm_plan(int n, size_t dbytes) {
  IluSm pl{};
  pl.ok = 0;
  if (n > 65535) return pl;
  const unsigned nwords = (n + 31) >> 5, nsum = (nwords + 31) >> 5;
  for (int lg = 12; lg >= 11; --lg) {
    const unsigned HS = 1u << lg, maxc = min((int)(HS / 2), kMaxRowNZ);
    unsigned o = 0;
    pl.o_bits = o; o += 4u * pad4(nwords);
    pl.o_sum = o; o += 4u * pad4(nsum);
    pl.o_ip = o; o += pad16(2 * n);
    pl.o_hkey = o; o += 4u * HS;
    pl.o_hidx = o; o += 2u * HS;
    pl.o_hslot = o; o += pad16(2 * maxc);
    pl.o_wv = o; o += pad16((int)sizeof(T) * maxc);
    if (o > dbytes) continue;
    pl.ok = 1; pl.HS = (int)HS; pl.lgHS = lg; pl.maxc = (int)maxc;
    // U-row cache: inverse diagonals, lengths and row offsets, then rows of (column, value)
    pl.o_meta = o;
    const unsigned mo = o + pad16((int)sizeof(T) * n);
    pl.o_len = mo;
    pl.o_uoff = mo + pad16(2 * n);
    pl.o_cc = pl.o_uoff + 4u * pad4(n + 1);
    pl.cache = 0;
    if (pl.o_cc + 64u * (4u + sizeof(T)) <= dbytes) {
      pl.cache = 1;
      pl.ucap = (unsigned)((dbytes - pl.o_cc) / (4u + sizeof(T))) & ~3u;
    }
    return pl;
  }
  return pl;
}

template <typename T>
__device__ __noinline__ int ilutp_warp_hash(const Walker& w, const Params& P, Shared& sh, const IluSm pl,
                                            int* npiv_out, double* nnz_out, int* p_out) {
  const int n = w.n, lane = threadIdx.x & 31, cap = w.cap, capLU = w.capLU;
  unsigned char* dsm = dyn_smem();
  unsigned* lbits = (unsigned*)(dsm + pl.o_bits);
  unsigned* lsum = (unsigned*)(dsm + pl.o_sum);
  unsigned short* ip = (unsigned short*)(dsm + pl.o_ip);
  int* hkey = (int*)(dsm + pl.o_hkey);
  unsigned short* hidx = (unsigned short*)(dsm + pl.o_hidx);
  unsigned short* hslot = (unsigned short*)(dsm + pl.o_hslot);
  T* wv = (T*)(dsm + pl.o_wv);
  const bool cache = pl.cache != 0;
  T* mdinv = (T*)(dsm + pl.o_meta);                  // cache: 1 / u_rr per row
  unsigned short* mlen = (unsigned short*)(dsm + pl.o_len);
  int* uoff = (int*)(dsm + pl.o_uoff);               // cache: row offset, or -1
  int* ucc = (int*)(dsm + pl.o_cc);
  T* ucv = (T*)(ucc + pl.ucap);
  const int ucap = cache ? (int)pl.ucap : 0;
  int ufill = 0;
  const int HS = pl.HS, hmask = HS - 1, hshift = 32 - pl.lgHS, MAXC = pl.maxc;
  const int nwords = (n + 31) >> 5, nsum = (nwords + 31) >> 5;
  for (int i = lane; i < nwords; i += 32) lbits[i] = 0u;
  for (int i = lane; i < nsum; i += 32) lsum[i] = 0u;
  for (int i = lane; i < HS; i += 32) hkey[i] = -1;
  for (int i = lane; i < n; i += 32) { w.perm[i] = i; ip[i] = (unsigned short)i; w.lev_l[i] = 0; }
  __syncwarp();
  int p = P.lfil_extra;
  if (p < 0) {
    long long tot = 0;
    for (int i = lane; i < n; i += 32) tot += w.a_len[i];
    tot = warp_sum_ll(tot);
    p = (int)((tot + 2LL * n - 1) / (2LL * n));  // ceil(avg nnz per row / 2)
  }
  p = min(p, (capLU - 2) / 2);
  const int pk = max(0, min(p, capLU - 2 - cap));
  int flags = 0, npiv = 0;
  long long n_elim = 0, n_cand = 0;
  double nnz = 0.0;
  auto hash_of = [&](int f) -> int { return (int)(((unsigned)f * 0x9E3779B1u) >> hshift); };
  // index of label f in the working row, or -1 (every lane the same)
  auto find = [&](int f) -> int {
    int h = hash_of(f);
    for (int probe = 0; probe < HS; ++probe) {
      const int k = hkey[h];
      if (k == f) { const int t = hidx[h]; return t == 0xFFFF ? -1 : t; }
      if (k == -1) return -1;
      h = (h + 1) & hmask;
    }
    return -1;
  };
  for (int r = 0; r < n; ++r) {
    const int part = w.part_of_row[r];
    const int len = w.a_len[part];
    const int* ac = w.a_col + (size_t)part * cap;
    const double* av = w.a_val + (size_t)part * cap;
    double ss = 0.0;
    int nl = 0, nu = 0;
    for (int t = lane; t < len; t += 32) {  // distinct labels: plain inserts
      const int f = ip[ac[t]];
      const double v = av[t];
      int h = hash_of(f);
      for (int probe = 0; probe < HS; ++probe) {
        if (atomicCAS(&hkey[h], -1, f) == -1) break;
        h = (h + 1) & hmask;
      }
      hidx[h] = (unsigned short)t;
      hslot[t] = (unsigned short)h;
      sh.nz[t] = f;
      wv[t] = (T)v;
      ss += v * v;
      nl += f < r;
      nu += f > r;
      if (f < r) {
        atomicOr(&lbits[f >> 5], 1u << (f & 31));
        atomicOr(&lsum[f >> 10], 1u << ((f >> 5) & 31));
      }
    }
    ss = warp_sum(ss);
    nl = warp_sum_int(nl);
    nu = warp_sum_int(nu);
    int cnt = len;
    const double norm = sqrt(ss);
    const T thr = (T)(P.drop_tol * norm);
    __syncwarp();
    // --- elimination with the previous U rows, in increasing label order ---
    int last = -1;
    for (;;) {
      int best = 0x7fffffff;
      __syncwarp();
      {
        // next pending label > last: first the rest of last's word, then the summary
        const int w0 = (last + 1) >> 5;
        const unsigned cur = w0 < nwords ? lbits[w0] & (0xffffffffu << ((last + 1) & 31)) : 0u;
        if (cur) {
          best = (w0 << 5) + __ffs(cur) - 1;
        } else {
          const int s0 = (w0 + 1) >> 5;  // summary word holding bitmap word w0 + 1
          for (int sb = s0; sb < nsum && best == 0x7fffffff; sb += 32) {
            const int si = sb + lane;
            unsigned sv = si < nsum ? lsum[si] : 0u;
            if (si == s0) sv &= 0xffffffffu << ((w0 + 1) & 31);
            const unsigned any = __ballot_sync(0xffffffffu, sv != 0u);
            if (any) {
              const int src = __ffs(any) - 1;
              const unsigned svs = __shfl_sync(0xffffffffu, sv, src);
              const int word = ((sb + src) << 5) + __ffs(svs) - 1;
              best = (word << 5) + __ffs(lbits[word]) - 1;
            }
          }
        }
      }
      if (best >= r) break;
      last = best;
      ++n_elim;
      // the U row of best: header and first 64 slots in one round trip (or the cache)
      const int ub = cache ? uoff[best] : -1;
      T dinv;
      int ul;
      int c0 = 0, c1 = 0;
      T v0 = 0, v1 = 0;
      if (ub >= 0) {
        dinv = mdinv[best];
        ul = mlen[best];
        if (lane < ul) { c0 = ucc[ub + lane]; v0 = ucv[ub + lane]; }
        if (lane + 32 < ul) { c1 = ucc[ub + lane + 32]; v1 = ucv[ub + lane + 32]; }
      } else {
        const size_t rb = (size_t)best * capLU;
        const double2 hd = w.u_head[best];
        if (lane < capLU) { c0 = w.u_col[rb + lane]; v0 = (T)w.u_val64[rb + lane]; }
        if (lane + 32 < capLU) { c1 = w.u_col[rb + lane + 32]; v1 = (T)w.u_val64[rb + lane + 32]; }
        dinv = (T)hd.x;
        ul = (int)hd.y;
      }
      const int tb = find(best);
      const T wk = wv[tb] * dinv;
      __syncwarp();
      if (fabs(wk) < thr) {
        if (lane == 0) wv[tb] = (T)0;  // dropped multiplier
        continue;
      }
      if (lane == 0) wv[tb] = wk;
      for (int base = 0; base < ul; base += 32) {
        const int t = base + lane;
        const bool valid = t < ul;
        int f = 0, h = 0, ex = -1;
        T v = 0;
        bool ins = false;
        if (valid) {
          int c;
          if (base == 0) { c = c0; v = v0; }
          else if (base == 32) { c = c1; v = v1; }
          else if (ub >= 0) { c = ucc[ub + t]; v = ucv[ub + t]; }
          else { c = w.u_col[(size_t)best * capLU + t]; v = (T)w.u_val64[(size_t)best * capLU + t]; }
          f = ip[c];
          h = hash_of(f);
          for (int probe = 0; probe < HS; ++probe) {
            const int k = hkey[h];
            if (k == f) { ex = hidx[h]; break; }
            if (k == -1) {
              const int old = atomicCAS(&hkey[h], -1, f);
              if (old == -1) { ins = true; break; }
              if (old == f) { ex = hidx[h]; break; }
            }
            h = (h + 1) & hmask;
          }
        }
        const unsigned nm = __ballot_sync(0xffffffffu, ins);
        const int slot_i = cnt + __popc(nm & lanemask_lt());
        if (ins) {
          if (slot_i < MAXC) {
            hidx[h] = (unsigned short)slot_i;
            hslot[slot_i] = (unsigned short)h;
            sh.nz[slot_i] = f;
            wv[slot_i] = -wk * v;
            if (f < r) {
              atomicOr(&lbits[f >> 5], 1u << (f & 31));
              atomicOr(&lsum[f >> 10], 1u << ((f >> 5) & 31));
            }
          } else {
            hidx[h] = 0xFFFF;  // over capacity: the factorisation is flagged unusable
          }
        } else if (valid && ex >= 0 && ex != 0xFFFF) {
          wv[ex] -= wk * v;
        }
        cnt += __popc(nm);
        __syncwarp();
      }
      if (cnt > MAXC) { flags |= 2; cnt = MAXC; }
    }
    n_cand += cnt;
    // --- L part: keep the nl + p largest multipliers ---
    T* selv = reinterpret_cast<T*>(sh.selV);
    int cL = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int t = base + lane;
      bool c = false;
      int f = 0;
      T v = 0;
      if (t < cnt) { f = sh.nz[t]; v = wv[t]; c = f < r && v != (T)0; }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      const int slot = cL + __popc(m & lanemask_lt());
      if (c && slot < kMaxSel) { sh.selF[slot] = f; selv[slot] = v; }
      cL += __popc(m);
    }
    if (cL > kMaxSel) { flags |= 2; cL = kMaxSel; }
    __syncwarp();
    const int keepL = nl + pk;
    select_topk<T>(sh, cL, keepL);
    int nL = 0, levmax = -1;
    for (int base = 0; base < cL; base += 32) {
      const int e = base + lane;
      const bool k = e < cL && sh.selK[e];
      const unsigned m = __ballot_sync(0xffffffffu, k);
      const int slot = nL + __popc(m & lanemask_lt());
      if (k && slot < capLU) {
        w.l_col[(size_t)r * capLU + slot] = sh.selF[e];
        w.l_val64[(size_t)r * capLU + slot] = (double)selv[e];
        levmax = max(levmax, w.lev_l[sh.selF[e]]);
      }
      nL += __popc(m);
    }
    levmax = warp_max_int(levmax);
    if (nL > capLU) { flags |= 2; nL = capLU; }
    __syncwarp();
    // --- U part: entries above threshold, keep the nu + p largest ---
    const int td = find(r);
    T dval = td >= 0 ? wv[td] : (T)0;
    int cU = 0;
    for (int base = 0; base < cnt; base += 32) {
      const int t = base + lane;
      bool c = false;
      int f = 0;
      T v = 0;
      if (t < cnt) { f = sh.nz[t]; v = wv[t]; c = f > r && fabs(v) >= thr && v != (T)0; }
      const unsigned m = __ballot_sync(0xffffffffu, c);
      const int slot = cU + __popc(m & lanemask_lt());
      if (c && slot < kMaxSel) { sh.selF[slot] = f; selv[slot] = v; }
      cU += __popc(m);
    }
    if (cU > kMaxSel) { flags |= 2; cU = kMaxSel; }
    __syncwarp();
    const int keepU = nu + pk;
    select_topk<T>(sh, cU, keepU);
    bool mykeep[kMaxSel / 32];
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      mykeep[q] = e < cU && sh.selK[e];
    }
    __syncwarp();
    // pivot: the largest kept U entry (ties: smaller label)
    T bv = 0;
    int bf = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      if (mykeep[q]) {
        const T v = fabs(selv[e]);
        const int f = sh.selF[e];
        if (v > bv || (v == bv && f < bf)) { bv = v; bf = f; }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      const int f2 = __shfl_xor_sync(0xffffffffu, bf, o);
      if (v2 > bv || (v2 == bv && f2 < bf)) { bv = v2; bf = f2; }
    }
    int jm = -1;
    if (bf != 0x7fffffff && (T)P.permtol * bv > fabs(dval)) jm = bf;
    T newdiag = dval;
    if (jm >= 0) {
      // the column labelled jm becomes the diagonal; the old diagonal value moves
      // to label jm (a U-part entry, or nothing if it was zero)
      newdiag = wv[find(jm)];
      if (lane == 0) {
        const int cr = w.perm[r], cj = w.perm[jm];
        w.perm[r] = cj; w.perm[jm] = cr;
        ip[cj] = (unsigned short)r; ip[cr] = (unsigned short)jm;
      }
      ++npiv;
    }
    __syncwarp();
    int nU = 0;
#pragma unroll
    for (int q = 0; q < kMaxSel / 32; ++q) {
      const int e = q * 32 + lane;
      bool k = mykeep[q];
      T v = 0;
      int f = 0;
      if (k) {
        f = sh.selF[e];
        v = selv[e];
        if (f == jm) { v = dval; k = dval != (T)0; }
      }
      const unsigned m = __ballot_sync(0xffffffffu, k);
      const int slot = nU + __popc(m & lanemask_lt());
      if (k && slot < capLU) {
        const int oc = w.perm[f];  // original column label
        w.u_col[(size_t)r * capLU + slot] = oc;
        w.u_val64[(size_t)r * capLU + slot] = (double)v;
        if (cache && ufill + slot < ucap) { ucc[ufill + slot] = oc; ucv[ufill + slot] = v; }
      }
      nU += __popc(m);
    }
    if (nU > capLU) { flags |= 2; nU = capLU; }
    if (newdiag == 0.0) {
      newdiag = (1e-4 + P.drop_tol) * (norm > 0.0 ? norm : 1.0);
      flags |= 1;
    }
    if (lane == 0) {
      const T di = (T)(1.0 / newdiag);
      w.l_len[r] = nL;
      w.u_len[r] = nU;
      w.u_dinv64[r] = (double)di;
      w.u_head[r] = make_double2((double)di, (double)nU);
      w.lev_l[r] = levmax + 1;
      if (cache) {
        mdinv[r] = di;
        mlen[r] = (unsigned short)nU;
        uoff[r] = ufill + nU <= ucap ? ufill : -1;
      }
    }
    if (cache && ufill + nU <= ucap) ufill += nU;
    nnz += (double)(nL + nU + 1);
    // clear the working row (and the pending-label bitmaps)
    for (int t = lane; t < cnt; t += 32) {
      const int f = sh.nz[t];
      hkey[hslot[t]] = -1;
      if (f < r) { lbits[f >> 5] = 0u; lsum[f >> 10] = 0u; }
    }
    if (flags & 2)  // keys past the capacity have no slot record: clear the whole table
      for (int i = lane; i < HS; i += 32) hkey[i] = -1;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) w.iperm[i] = ip[i];
  __syncwarp();
  if (lane == 0) { w.ctl->ilu_rows += n; w.ctl->ilu_elims += n_elim; w.ctl->ilu_cand += n_cand; }
  *npiv_out = npiv;
  *nnz_out = nnz;
  *p_out = p;
  return flags;
}

// ---------------------------------------------------------------------------
// Level-ordered chunk stream of one triangular factor, consumed by the staged
// solve.  Consecutive levels are packed into a chunk (one segment each) while it
// stays within the slot size and kMaxSeg segments; a level larger than a slot is
// split over chunks.  The rows of a segment are independent.  Returns the number of
// chunks.  Block-wide (packing by thread 0: sequential over levels, and over rows
// only inside levels that must be split).
// ---------------------------------------------------------------------------
// Grouped form (expanded = true): the segments are groups of consecutive levels and the
// rows are the expanded rows of expand_groups (no diagonal array; chunk header .w = 1).
template <typename T>
__device__ int build_stream(const Walker& w, const Params& P, bool upper, int nlev, Shared& sh,
                            bool expanded = false) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int* lptr = expanded ? w.gptr : (upper ? w.u_lvl_ptr : w.l_lvl_ptr);
  const int* rows = upper ? w.u_lvl_rows : w.l_lvl_rows;
  const int* len = expanded ? w.ex_len : (upper ? w.u_len : w.l_len);
  const int* colv = expanded ? w.ex_col : (upper ? w.u_col : w.l_col);
  const double* valv = expanded ? w.ex_val : (upper ? w.u_val64 : w.l_val64);
  int2* tab = upper ? w.uchunk : w.lchunk;
  unsigned char* stream = upper ? w.ustream : w.lstream;
  const int tsz = (int)sizeof(T), capLU = expanded ? w.exmax : w.capLU;
  const bool with_dv = upper && !expanded;
  auto cbytes = [&](int ns, int r, int e) {
    return expanded ? chunk_bytes_grouped(ns, r, e, tsz) : chunk_bytes(ns, r, e, tsz, with_dv);
  };
  const int SB = P.slot_bytes;
  const int nct = nt - 32;  // consumer threads of the solve
  // entries per level and the level's lane-group size (warp per level).  The group size
  // is a property of the level, not of the chunk a piece of it lands in, so the rounding
  // of every row is independent of the slot size.  Enough lanes for <= P.lane_entries
  // entries per lane on the level's longest row (the level barrier waits for it), while
  // the rows still fit the consumer threads once.  Few entries a lane (FP32: 2) keep the
  // dependent chain short; FP64 takes more (8), because every lane-group reduction step
  // is an FP64 add and GB300's FP64 pipe issues few per clock.  Packed as
  // entries | gs << 28 (entries < 2^28 for K <= 64).
  for (int lev = wid; lev < nlev; lev += nw) {
    int e = 0, ml = 0;
    for (int q = lptr[lev] + lane; q < lptr[lev + 1]; q += 32) {
      const int L = len[rows[q]];
      e += L;
      ml = max(ml, L);
    }
    e = warp_sum_int(e);
    ml = warp_max_int(ml);
    const int lr = lptr[lev + 1] - lptr[lev];
    int gs = 0;
    while (gs < 5 && (P.lane_entries << gs) < ml && (lr << (gs + 1)) <= nct) ++gs;
    if (lane == 0) w.lvl_nchunk[lev] = e | (gs << 28);
  }
  __syncthreads();
  if (tid == 0) {
    int nch = 0, nseg = 0;
    int cs = 0, cr = 0, ce = 0;  // open chunk: segments, rows, entries
    int c_seg0 = 0;
    for (int lev = 0; lev < nlev; ++lev) {
      int q = lptr[lev];
      const int qe = lptr[lev + 1];
      const int lr = qe - q, le = w.lvl_nchunk[lev] & ((1 << 28) - 1);
      // levels of at most P.warp_rows rows are solved by one warp alone, with no barrier
      // among the solving warps; the segment records 1 + log2 of that warp's lanes per row
      // (0: all warps).  Decided per level, so that pieces of a level split over chunks
      // round alike.
      const int gsl = w.lvl_nchunk[lev] >> 28;
      int gw = gsl;
      while (gw > 0 && (lr << gw) > 32) --gw;
      const int wmode = (!expanded && lr <= P.warp_rows && (lr << gw) <= 32) ? gw + 1 : 0;
      const int lgs = gsl | (wmode << 8);
      if (cs < kMaxSeg && cbytes(cs + 1, cr + lr, ce + le) <= SB) {
        w.seg_meta[nseg++] = make_int4(q, lr, le, lgs);  // the whole level joins the open chunk
        ++cs; cr += lr; ce += le;
        continue;
      }
      while (q < qe) {  // close the open chunk if any, then pieces of this level
        if (cs > 0 && (cs == kMaxSeg || cbytes(cs + 1, cr + 1, ce + len[rows[q]]) > SB)) {
          w.chunk_meta[nch] = make_int4(c_seg0, cs, cr, ce);
          w.lvl_cur[nch] = cbytes(cs, cr, ce);
          ++nch; c_seg0 = nseg; cs = 0; cr = 0; ce = 0;
        }
        const int q0 = q;
        int pr = 0, pe = 0;
        while (q < qe) {
          const int L = len[rows[q]];
          if ((cr + pr) > 0 && cbytes(cs + 1, cr + pr + 1, ce + pe + L) > SB) break;
          ++pr; pe += L; ++q;
        }
        w.seg_meta[nseg++] = make_int4(q0, pr, pe, lgs);
        ++cs; cr += pr; ce += pe;
        if (q < qe) {  // the slot is full: close it
          w.chunk_meta[nch] = make_int4(c_seg0, cs, cr, ce);
          w.lvl_cur[nch] = cbytes(cs, cr, ce);
          ++nch; c_seg0 = nseg; cs = 0; cr = 0; ce = 0;
        }
      }
    }
    if (cs > 0) {
      w.chunk_meta[nch] = make_int4(c_seg0, cs, cr, ce);
      w.lvl_cur[nch] = cbytes(cs, cr, ce);
      ++nch;
    }
    sh.iflag[2] = nch;
  }
  __syncthreads();
  const int nch_total = sh.iflag[2];
  for (int c = tid; c < nch_total; c += nt) tab[c].y = w.lvl_cur[c];
  __syncthreads();
  block_scan_inplace(w.lvl_cur, nch_total, sh);
  for (int c = tid; c < nch_total; c += nt) tab[c].x = w.lvl_cur[c];
  __syncthreads();
  // fill the chunks, one warp per chunk
  if (expanded) {
    for (int c = wid; c < nch_total; c += nw) {
      const int4 cm = w.chunk_meta[c];
      const int seg0 = cm.x, nseg = cm.y, nr = cm.z, ne = cm.w;
      unsigned char* base = stream + tab[c].x;
      int4* seg = (int4*)(base + kChunkHdr);
      int4* desc = (int4*)(base + kChunkHdr + 16 * nseg);
      unsigned char* ent = base + kChunkHdr + 16 * nseg + 16 * nr;
      if (lane == 0) *(int4*)base = make_int4(nseg, nr, ne, 1);
      if (lane < kMaxSlots)
        ((int2*)(base + 16))[lane] = c + 1 + lane < nch_total ? tab[c + 1 + lane] : make_int2(0, 0);
      int rbase = 0, carry = 0;
      for (int sgi = 0; sgi < nseg; ++sgi) {
        const int4 sm = w.seg_meta[seg0 + sgi];
        const int q0 = sm.x, sr = sm.y;
        if (lane == 0) seg[sgi] = make_int4(rbase, sr, sm.w & 0xff, 0);
        for (int b0 = 0; b0 < sr; b0 += 32) {
          const int i = b0 + lane;
          const int r = i < sr ? rows[q0 + i] : 0;
          const int L = i < sr ? len[r] : 0;
          int inc = L;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
          }
          if (i < sr) desc[rbase + i] = make_int4(r, carry + inc - L, carry + inc, 0);
          carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        rbase += sr;
      }
      __syncwarp();
      for (int i = 0; i < nr; ++i) {
        const int4 d = desc[i];
        const int r = d.x, b = d.y, L = d.z - d.y;
        for (int t = lane; t < L; t += 32) {
          const int col = colv[(size_t)r * capLU + t];
          const double val = valv[(size_t)r * capLU + t];
          if (tsz == 4) {
            reinterpret_cast<float2*>(ent)[b + t] = make_float2(__int_as_float(col), (float)val);
          } else {
            reinterpret_cast<int*>(ent)[b + t] = col;
            reinterpret_cast<double*>(ent + pad16(4 * ne))[b + t] = val;
          }
        }
      }
    }
    __syncthreads();
    return nch_total;
  }
  for (int c = wid; c < nch_total; c += nw) {
    const int4 cm = w.chunk_meta[c];
    const int seg0 = cm.x, nseg = cm.y, nr = cm.z, ne = cm.w;
    unsigned char* base = stream + tab[c].x;
    int4* seg = (int4*)(base + kChunkHdr);
    int* rws = (int*)(base + kChunkHdr + 16 * nseg);
    int* st = rws + pad4(nr);
    int* cl = st + pad4(nr + 1);
    T* vl = (T*)(cl + pad4(ne));
    T* dv = (T*)((unsigned char*)vl + pad16(tsz * ne));
    if (lane == 0) *(int4*)base = make_int4(nseg, nr, ne, expanded ? 1 : 0);
    if (lane < kMaxSlots) ((int2*)(base + 16))[lane] = c + 1 + lane < nch_total ? tab[c + 1 + lane] : make_int2(0, 0);
    int rbase = 0, carry = 0;
    for (int sgi = 0; sgi < nseg; ++sgi) {
      const int4 sm = w.seg_meta[seg0 + sgi];
      const int q0 = sm.x, sr = sm.y;
      if (lane == 0) seg[sgi] = make_int4(rbase, sr, sm.w & 0xff, sm.w >> 8);
      for (int b0 = 0; b0 < sr; b0 += 32) {
        const int i = b0 + lane;
        const int r = i < sr ? rows[q0 + i] : 0;
        const int L = i < sr ? len[r] : 0;
        int inc = L;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += v;
        }
        if (i < sr) {
          rws[rbase + i] = r;
          st[rbase + i] = carry + inc - L;
          if (with_dv) dv[rbase + i] = (T)w.u_dinv64[r];
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);
      }
      rbase += sr;
    }
    if (lane == 0) st[nr] = carry;
    __syncwarp();
    for (int i = 0; i < nr; ++i) {
      const int r = rws[i];
      const int b = st[i], L = st[i + 1] - b;
      for (int t = lane; t < L; t += 32) {
        cl[b + t] = colv[(size_t)r * capLU + t];
        vl[b + t] = (T)valv[(size_t)r * capLU + t];
      }
    }
  }
  __syncthreads();
  return nch_total;
}

// ---------------------------------------------------------------------------
// Grouped triangular solves (a partitioned inverse of the factor).  Consecutive levels
// of L (of U) are merged into groups of at most P.tri_group levels; every row of a group
// is expanded by substituting the rows of the same group it depends on, so that it
// reads only the input vector v and solution entries of earlier groups:
//   L:  y_r = v_r - sum_c L_rc y_c          ->  y_r = sum_q a_rq v_q + sum_{c earlier} b_rc y_c
//   U:  x_r = (y_r - sum_c U_rc x_c) / U_rr  ->  x_r = sum_q a_rq y_q + sum_{c earlier} b_rc x_c
// (q over the row and its ancestors inside the group).  The rows of a group are then
// independent, and the solve needs one barrier per group instead of one per level.  The
// operator is the same as the level-by-level substitution in exact arithmetic (the
// coefficients are formed in FP64 and rounded once to the working precision).  Indices
// of the expanded rows are offsets from the solution vector: c in [0, n) the solution
// entry c; the input entry q at n + q for L (the input vector follows the solution) and
// at q - n for U (it precedes it: the L solution is U's input).  A level joins the open
// group only while every expanded row of it stays within w.exmax entries; otherwise it
// starts a new group.
// Block-wide; one warp per row with a hash accumulator of 2 exmax slots in the dynamic
// shared memory (idle after the factorisation).  Writes w.gptr (row pointer of each
// group into the level-ordered rows), w.ex_len/ex_col/ex_val; returns the group count.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int expand_groups(const Walker& w, const Params& P, bool upper, int nlev, Shared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int n = w.n, capLU = w.capLU, EX = w.exmax;
  const int* lptr = upper ? w.u_lvl_ptr : w.l_lvl_ptr;
  const int* rows = upper ? w.u_lvl_rows : w.l_lvl_rows;
  const int* flen = upper ? w.u_len : w.l_len;
  const int* fcol = upper ? w.u_col : w.l_col;
  const double* fval = upper ? w.u_val64 : w.l_val64;
  const int* lev = upper ? w.lev_u : w.lev_l;
  const int hs = group_hash_slots(EX);  // per-warp table: at most half full
  const int hmask = hs - 1;
  constexpr int kEmpty = (int)0x80000000;  // keys are offsets in [-n, 2n)
  const int in_off = upper ? -n : n;
  int* hkey = reinterpret_cast<int*>(dyn_smem()) + (size_t)wid * hs * 3;  // keys, then values (8-byte aligned)
  double* hval = reinterpret_cast<double*>(hkey + hs + (hs & 1));
  auto add = [&](int key, double v, int& cnt, bool& over, bool active) {
    // lanes with active = true add distinct keys; returns the updated count (uniform)
    bool ins = false;
    int h = 0;
    if (active) {
      h = (int)(((unsigned)key * 0x9E3779B1u) >> 7) & hmask;
      for (int probe = 0; probe < hs; ++probe) {
        const int k = hkey[h];
        if (k == key) { hval[h] += v; break; }
        if (k == kEmpty) {
          const int old = atomicCAS(&hkey[h], kEmpty, key);
          if (old == kEmpty) { hval[h] = v; ins = true; break; }
          if (old == key) { hval[h] += v; break; }
        }
        h = (h + 1) & hmask;
      }
    }
    cnt += __popc(__ballot_sync(0xffffffffu, ins));
    if (cnt > EX) over = true;
    __syncwarp();
  };
  // expand the rows of level lv with the open group starting at level g; returns true
  // (block-uniform) when a row exceeded exmax entries
  auto expand_level = [&](int lv, int g) -> bool {
    bool any_over = false;
    for (int q = lptr[lv] + wid; q < lptr[lv + 1]; q += nw) {
      const int r = rows[q];
      for (int i = lane; i < hs; i += 32) hkey[i] = kEmpty;
      __syncwarp();
      const double d = upper ? w.u_dinv64[r] : 1.0;
      int cnt = 0;
      bool over = false;
      add(in_off + r, d, cnt, over, lane == 0);
      const int L = flen[r];
      const int* rc = fcol + (size_t)r * capLU;
      const double* rv = fval + (size_t)r * capLU;
      for (int t0 = 0; t0 < L; t0 += 32) {  // dependencies on earlier groups
        const int t = t0 + lane;
        const bool act = t < L && lev[rc[t]] < g;
        add(act ? rc[t] : 0, act ? -d * rv[t] : 0.0, cnt, over, act);
      }
      for (int t = 0; t < L && !over; ++t) {  // dependencies inside the group: substitute
        const int c = rc[t];
        if (lev[c] < g) continue;
        const double coef = -d * rv[t];
        const int el = w.ex_len[c];
        const int* ec = w.ex_col + (size_t)c * EX;
        const double* ev = w.ex_val + (size_t)c * EX;
        for (int e0 = 0; e0 < el; e0 += 32) {
          const int e = e0 + lane;
          add(e < el ? ec[e] : 0, e < el ? coef * ev[e] : 0.0, cnt, over, e < el);
        }
      }
      // write the expanded row (slot order)
      int outc = 0;
      for (int i0 = 0; i0 < hs; i0 += 32) {
        const int i = i0 + lane;
        const bool k = !over && hkey[i] != kEmpty;
        const unsigned m = __ballot_sync(0xffffffffu, k);
        const int slot = outc + __popc(m & lanemask_lt());
        if (k && slot < EX) {
          w.ex_col[(size_t)r * EX + slot] = hkey[i];
          w.ex_val[(size_t)r * EX + slot] = hval[i];
        }
        outc += __popc(m);
      }
      if (lane == 0) w.ex_len[r] = over ? 0 : min(outc, EX);
      any_over |= over;
      __syncwarp();
    }
    const int o = block_max_int(any_over ? 1 : 0, sh);  // ends synchronised
    return o != 0;
  };
  int g0 = 0, ngrp = 0;
  if (tid == 0) w.gptr[0] = 0;
  for (int lv = 0; lv < nlev; ++lv) {
    const bool join = lv > 0 && lv - g0 < P.tri_group;
    bool newg = !join;
    if (join && expand_level(lv, g0)) newg = true;
    if (newg) {
      if (lv > 0) {
        ++ngrp;
        if (tid == 0) w.gptr[ngrp] = lptr[lv];
      }
      g0 = lv;
      expand_level(lv, lv);
    }
  }
  ++ngrp;
  if (tid == 0) w.gptr[ngrp] = lptr[nlev];
  __syncthreads();
  return ngrp;
}

// Block-wide: relabel U columns to factor labels, compute U levels (warp 0,
// reverse order) and pack both level sets (counting sort by level).
template <typename T>
__device__ __noinline__ void relabel_and_levels(const Walker& w, const Params& P, Shared& sh) {
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
  if (tid == 0) { w.ctl->nlev_l = nll; w.ctl->nlev_u = nlu; }
  __syncthreads();
  int ncl, ncu;
  if (grouped_solves<T>(w, P)) {
    const int gl = expand_groups<T>(w, P, false, nll, sh);
    ncl = build_stream<T>(w, P, false, gl, sh, true);
    const int gu = expand_groups<T>(w, P, true, nlu, sh);
    ncu = build_stream<T>(w, P, true, gu, sh, true);
    if (tid == 0) { w.ctl->ngrp_l = gl; w.ctl->ngrp_u = gu; }
  } else {
    ncl = build_stream<T>(w, P, false, nll, sh);
    ncu = build_stream<T>(w, P, true, nlu, sh);
    if (tid == 0) { w.ctl->ngrp_l = nll; w.ctl->ngrp_u = nlu; }
  }
  if (tid == 0) {
    w.ctl->nchunk_l = ncl;
    w.ctl->nchunk_u = ncu;
    w.ctl->stream_bytes = (ncl ? (long long)w.lchunk[ncl - 1].x + w.lchunk[ncl - 1].y : 0) +
                          (ncu ? (long long)w.uchunk[ncu - 1].x + w.uchunk[ncu - 1].y : 0);
  }
  fence_proxy_async_global();  // the streams are read next by bulk (async-proxy) copies
  __syncthreads();
}

// Full (re)factorisation: optional reorder, ILUTP, levels; clears the update chain.
// Block-wide.  Returns the ILUTP flags.
template <typename T>
__device__ __noinline__ int factor_block(const Walker& w, const Params& P, Shared& sh, bool reorder) {
  const long long t0 = clock64();
  if (reorder) {
    reorder_block(w, sh);
    if (threadIdx.x == 0) w.ctl->cyc[PH_REORDER] += clock64() - t0;
  }
  if (threadIdx.x < 32) {
    int npiv = 0, p = 0;
    double nnz = 0.0;
    for (int r = threadIdx.x; r < w.n; r += 32) w.lev_u[r] = 0;
    const long long ti = clock64();
    int fl;
    const IluSm pl64 = ilu_sm_plan<double>(w.n, (size_t)P.dsm_bytes);
    const IluSm plT = ilu_sm_plan<T>(w.n, (size_t)P.dsm_bytes);
    // the shared-memory variant where the dense working row does not fit in shared memory
    // (about n > 6000 with one walker CTA per SM); below that the dense row is in shared
    // memory too and, with its U-row cache, the faster of the two
    const bool dense_row_in_smem = 4 * (size_t)(pad4((w.n + 31) >> 5) + pad4((((w.n + 31) >> 5) + 31) >> 5)) +
                                       16 + (size_t)16 * w.n <= (size_t)P.dsm_bytes;
    if (P.ilu_variant == 0 && !dense_row_in_smem && w.u_head != nullptr && (P.ilu64 ? pl64.ok : plT.ok))
      fl = P.ilu64 ? ilutp_warp_hash<double>(w, P, sh, pl64, &npiv, &nnz, &p)
                   : ilutp_warp_hash<T>(w, P, sh, plT, &npiv, &nnz, &p);
    else if (P.ilu_variant == 2 && w.u_head != nullptr && (P.ilu64 ? pl64.ok : plT.ok))  // forced (tests)
      fl = P.ilu64 ? ilutp_warp_hash<double>(w, P, sh, pl64, &npiv, &nnz, &p)
                   : ilutp_warp_hash<T>(w, P, sh, plT, &npiv, &nnz, &p);
    else
      fl = P.ilu64 ? ilutp_warp<double>(w, P, sh, &npiv, &nnz, &p) : ilutp_warp<T>(w, P, sh, &npiv, &nnz, &p);
    if (threadIdx.x == 0) w.ctl->cyc[PH_ILUTP] += clock64() - ti;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // scratch is reused by bulk copies
    if (threadIdx.x == 0) {
      sh.iflag[0] = fl;
      Ctl* c = w.ctl;
      c->last_pivots = npiv;
      c->nnz_LU = nnz;
      c->p_lfil = p;
      c->factorizations += 1;
      c->n_upd = 0;
      c->upd_nnz = 0;
      c->last_breakdown = fl & 1;
      c->fresh = reorder ? 1 : 0;  // a synchronous reorder + refactorisation of the current matrix
      c->af_epoch += 1;  // a background factorisation requested before this one is stale
    }
  }
  __syncthreads();
  const int fl = sh.iflag[0];
  const long long tl = clock64();
  relabel_and_levels<T>(w, P, sh);
  if (threadIdx.x == 0) w.ctl->cyc[PH_LEVELS] += clock64() - tl;
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int i = 0; i < w.n; ++i) tot += w.a_len[i];
    w.ctl->nnz_A = (double)tot;
    w.ctl->cyc[PH_FACTOR] += clock64() - t0;
  }
  __syncthreads();
  return fl;
}

}  // namespace vmc
