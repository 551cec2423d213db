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
//     triangular-solve dependency depth small; make_layout in vmc_capi.cu);
//   * ILUTP factors of A_p Q = L U (Sec. 3.2 Eq. 14) in fixed-capacity rows, the
//     column permutation perm/iperm, level sets and the chunk streams the triangular
//     solves read (two such factor sets when a second CTA refactors in the background);
//   * the chain of rank-one preconditioner updates (z_hat_s, u_s) of Sec. 3.2 Eq. 18
//     with the small matrix G[s][t] = u_s^T z_hat_t;
//   * the Krylov basis V and preconditioned vectors Zk of GMRES (Sec. 3.2 Eq. 15).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vmc {

constexpr int kMaxThreads = 256;  // largest walker CTA (two per SM with up to 128 registers a thread)
constexpr int kMaxM = 40;         // largest Krylov dimension
constexpr int kMaxRow = 256;      // largest Slater row (entries)
constexpr int kMaxU = 2 * kMaxRow;
constexpr int kMaxRowNZ = 2048;   // ILUTP working-row entries before dropping
constexpr int kMaxSel = 1024;     // ILUTP candidates of one triangle
constexpr int kMaxUpd = 128;      // longest preconditioner update chain
constexpr int kHistBins = 64;
constexpr int kSlotBytes = 8192;  // smallest ring slot (a slot holds the largest stream chunk)
constexpr int kMaxSlots = 8;      // ring depth (chunks in flight)
constexpr int kChunkHdr = 80;     // chunk header bytes: int4 + 8 next-chunk descriptors
constexpr int kMaxSeg = 32;       // levels (segments) per chunk at most
// phase indices of Ctl::cyc
enum : int { PH_BUILD = 0, PH_FIRST = 1, PH_REFINE = 2, PH_FACTOR = 3, PH_REORDER = 4, PH_COMMIT = 5, PH_STEP = 6,
             PH_TRI = 7, PH_CHAIN = 8, PH_SPMV = 9, PH_ORTH = 10, PH_RESID = 11, PH_ILUTP = 12, PH_LEVELS = 13, PH_TRIWAIT = 14,
             PH_TRIDATA = 15 };

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
  int nchunk_l, nchunk_u;
  int ngrp_l, ngrp_u;  // barriers of the triangular solves (groups; = levels when not grouped)
  long long stream_bytes;  // bytes of the L and U chunk streams (read by every preconditioner apply)
  double pend_r[3];
  double pend_ratio;
  double pend_grad[3], pend_lap;  // gradient / Laplacian at the pending position (when asked)
  double its_sum;
  long long its_cnt;
  long long proposals, accepts, solves, inner_its, first_its, outer_passes;
  long long reorders, reorder_monitor, reorder_noconv, reorder_slow, reorder_breakdown;
  long long refactors_updates, factorizations;
  double N_max_seen, N_sum;
  double nnz_A, nnz_LU;
  long long hist[kHistBins];
  long long cyc[16];  // clock64 cycles by phase (see vmc_stats.phase_cycles)
  double alg_bytes;   // compulsory (algorithmic) bytes moved by the solves, counted per phase
  long long ilu_rows, ilu_elims, ilu_cand;  // ILUTP rows, eliminations, working-row entries
  int upd_nnz;        // total nonzeros of the u vectors in the update chain
  // Background refactorisation (persistent engine with a factor CTA per walker).  The
  // solver uses factor set `active`; the factor CTA fills set af_target from a snapshot
  // of A taken when the chain held af_snap updates.
  int active;         // factor set in use (0 or 1)
  int af_state;       // 0 idle, 1 requested, 2 result ready (written with release order)
  int af_target;      // factor set being filled
  int af_snap;        // chain length at the snapshot
  int af_epoch;       // bumped by every factorisation on this controller
  int af_epoch_req;   // af_epoch when the request in flight was made
  int af_stop;        // launch id after which the factor CTA leaves
  int af_fail;        // the last background factorisation reported (bit 0 breakdown, bit 1 capacity)
  long long refactors_async, af_wait_cyc, af_factor_cyc;
  // 1 while the factors in use come from a synchronous reorder + refactorisation of the
  // current matrix (no move accepted and no background factors adopted since): a trigger
  // then cannot be helped by refactoring, which would reproduce the same factors
  int fresh;
  long long reorder_skipped;
  long long trig_its;  // iterations until the residual reached trig_rtol, summed over solves
  // position of the walker's chain after a budgeted advance: the next move is particle
  // pos_k of sweep pos_sweep (pos_valid = 0: particle 0 of the context's sweep counter)
  long long pos_sweep;
  int pos_k, pos_valid;
};

// Immutable-per-context description of one walker: sizes and device pointers.
struct Walker {
  int n, K, lattice, cap, capLU, m, mu;
  int mu4;                // row stride of the transposed z_hat store (mu rounded up to 4)
  int per;                // sites per cubic cell (1 sc, 2 bcc)
  double a, kappa, rc, rc2, L;
  const double* Z;        // n*3 orbital centres
  const int* col_of_orb;  // fixed column of each orbital
  const int* orb_of_col;
  double* R;              // n*3 positions by particle
  int* row_of_part;
  int* part_of_row;
  int* a_col; double* a_val; float* a_val32; int* a_len;
  int* l_col; double* l_val64; int* l_len;
  int* u_col; double* u_val64; int* u_len;
  double* u_dinv64;
  double2* u_head;        // per U row {1 / u_rr, length}, written by the shared-memory ILUTP
  // grouped triangular solves: expanded rows (exmax entries each) and group row pointers
  int exmax; int* ex_len; int* ex_col; double* ex_val; int* gptr;
  // level-ordered chunk streams of L and U for the staged triangular solves
  unsigned char* lstream; unsigned char* ustream;
  int2* lchunk; int2* uchunk;   // per chunk {byte offset, bytes}
  int4* chunk_meta;             // scratch per chunk {first segment, segments, rows, entries}
  int4* seg_meta;               // scratch per segment {first row in level order, rows, entries, 0}
  int* lvl_nchunk;              // scratch per level
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
  // dense engine (explicit inverse): B row-major n x n, two work vectors, pivots
  double* Bd; double* dcol; double* drow; int* dpiv;
  // background refactorisation: the same walker with the other factor set (nullptr when
  // the context has one set), and the factor CTA's views (factor set s, the snapshot of
  // A as its matrix, the shadow controller as its ctl)
  const Walker* alt;
  const Walker* fact[2];
  int set_id;
  int* snap_len; int* snap_col; double* snap_val; int* snap_part;
  double* snap_R; int* snap_rop;  // positions and row-of-particle at the snapshot
  Ctl* shadow;
};

// The view of walker w0 (factor set 0) that the solver uses now.
__device__ __forceinline__ const Walker& active_of(const Walker& w0) {
  return (w0.alt != nullptr && w0.ctl->active) ? *w0.alt : w0;
}

struct Params {
  double drop_tol, permtol;
  int lfil_extra, m, max_restarts, max_updates;
  double inner_rtol, ratio_tol, N_max, slow_factor;
  int ring_slots;   // shared-memory ring depth for the triangular-solve streams
  int y_smem;       // 1: the triangular-solve vector lives in shared memory
  int y_bytes;      // bytes reserved for it (multiple of 128)
  int slot_bytes;   // bytes of one ring slot = largest stream chunk (multiple of 16)
  int dsm_bytes;    // total dynamic shared memory (ILUTP scratch may use all of it)
  int ilu64;        // 1: the ILUTP working row is FP64 whatever the stored precision
  int af_lag;       // background refactorisation: accepts between a snapshot and its use (0: off)
  int af_reorder;   // 1: background refactorisations re-pair particles and orbitals first
  int step_limit;   // > 0: a sweep moves only particles 0 .. step_limit - 1 (autotuner trials)
  int tri_sf;       // 1: synchronisation-free triangular solves (two solve vectors in shared memory)
  int y_half;       // byte offset of the second solve vector (tri_sf)
  double trig_rtol; // controller: the solve converged if its residual reached this ...
  int trig_its;     // ... within this many GMRES iterations (all cycles)
  int ilu_variant;  // 0: auto (hash working row where the dense one misses shared memory); 1: dense; 2: hash
  int warp_rows;    // levels of at most this many rows: triangular-solve rows by one warp, no barrier
  int tri_group;    // > 1: grouped triangular solves, at most this many levels per group
  int lane_entries; // entries per lane the triangular solves' lane groups are sized for
  // budgeted advance of the persistent engine: the walkers claim moves one at a time from
  // *budget_ctr until budget_total are claimed (nullptr: fixed sweeps)
  unsigned long long* budget_ctr;
  long long budget_total;
};

// Shared memory of a walker CTA (static, < 48 KB).
struct __align__(16) Shared {
  unsigned long long bar[kMaxSlots];  // "full" mbarriers of the stream ring
  unsigned long long ebar[kMaxSlots]; // "empty" mbarriers (released by the consumer warps)
  int ring_seq;                       // chunks consumed so far in this launch
  union {
    struct {                          // GMRES
      double H[(kMaxM + 1) * kMaxM];
      double g[kMaxM + 1], cs[kMaxM], sn[kMaxM], y[kMaxM];
      double h1[kMaxM + 2], h2[kMaxM + 2];
    };
    struct {                          // ILUTP working row
      int nz[kMaxRowNZ];
      int selF[kMaxSel];
      double selV[kMaxSel];
      unsigned char selK[kMaxSel];    // top-k selection result per candidate
      int hist[64];                   // exponent histogram of the selection
      int bndE[256];                  // candidates of the boundary octave
    };
  };
  double red[40];
  double redv[33];
  int redi[33];
  double rnew[3];
  double aval[kMaxRow];
  int acol[kMaxRow];
  double uval[kMaxU];
  int ucol[kMaxU];
  double cupd[kMaxUpd];
  int alen, ulen;
  int iflag[12];
  double dflag[8];
};

// Grouped triangular solves (expand_groups): on when asked for, the walker has the
// scratch for the expanded rows, its two solve vectors fit the shared-memory solve area,
// and one hash accumulator per warp of the CTA fits the dynamic shared memory (else the
// level-by-level solve, in place on one vector).  Decided the same way at factorisation
// and solve.
__device__ __forceinline__ int group_hash_slots(int exmax) {
  int hs = 64;
  while (hs < 2 * exmax) hs <<= 1;
  return hs;
}
template <typename T>
__device__ __forceinline__ bool grouped_solves(const Walker& w, const Params& P) {
  return P.tri_group > 1 && w.ex_col != nullptr && P.y_smem &&
         2 * (size_t)w.n * sizeof(T) <= (size_t)P.y_bytes &&  // both solve vectors in shared memory
         (size_t)(blockDim.x >> 5) * 12u * (size_t)group_hash_slots(w.exmax) <= (size_t)P.dsm_bytes;
}

// ---- block-wide copies with several loads in flight per thread ---------------
// A plain loop `dst[i] = src[i]` between pointers that may alias issues each load only
// after the previous iteration's store, i.e. one memory latency per iteration; these
// issue kCopyBatch loads before their stores.
constexpr int kCopyBatch = 8;
template <typename T>
__device__ __forceinline__ void block_copy(T* dst, const T* src, int n) {
  const int nt = blockDim.x;
  for (int i0 = threadIdx.x; i0 < n; i0 += kCopyBatch * nt) {
    T v[kCopyBatch];
#pragma unroll
    for (int k = 0; k < kCopyBatch; ++k) {
      const int i = i0 + k * nt;
      v[k] = i < n ? src[i] : T(0);
    }
#pragma unroll
    for (int k = 0; k < kCopyBatch; ++k) {
      const int i = i0 + k * nt;
      if (i < n) dst[i] = v[k];
    }
  }
}
// dst[idx[i]] = src[i]
template <typename T>
__device__ __forceinline__ void block_scatter(T* dst, const int* idx, const T* src, int n) {
  const int nt = blockDim.x;
  for (int i0 = threadIdx.x; i0 < n; i0 += kCopyBatch * nt) {
    T v[kCopyBatch];
    int d[kCopyBatch];
#pragma unroll
    for (int k = 0; k < kCopyBatch; ++k) {
      const int i = i0 + k * nt;
      v[k] = i < n ? src[i] : T(0);
      d[k] = i < n ? idx[i] : 0;
    }
#pragma unroll
    for (int k = 0; k < kCopyBatch; ++k) {
      const int i = i0 + k * nt;
      if (i < n) dst[d[k]] = v[k];
    }
  }
}

// ---- dynamic shared memory, mbarriers and bulk (TMA) copies ----------------
__device__ __forceinline__ unsigned char* dyn_smem() {
  extern __shared__ __align__(128) unsigned char vmc_dsm[];
  return vmc_dsm;
}
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy completing on bar; dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// The same with an L2 eviction-priority policy (createpolicy): the chunk streams are
// re-read by every preconditioner apply and are asked to stay in L2 ahead of data read
// once per apply.
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                              unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of bar to complete; gives up after ~1 s (returns false).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  unsigned ok = 0;
  asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
               : "=r"(ok) : "r"(a), "r"(parity) : "memory");
  if (ok) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// Longest wait between the two CTAs of a walker pair (either side), in ns.
constexpr unsigned long long kPairWaitNs = 30ull * 1000000000ull;
// Wait (thread 0) until *state differs from `from`; returns the new value, or -1 after
// kPairWaitNs.
__device__ __forceinline__ int wait_state_change(const int* state, int from) {
  int v = ld_acquire(state);
  if (v != from) return v;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(1000);
    v = ld_acquire(state);
    if (v != from) return v;
    if (global_ns() - t0 > kPairWaitNs) return -1;
  }
}

// Byte layout of one stream chunk (all offsets multiples of 16): a run of consecutive
// levels ("segments"; a level too large for one slot is split over several chunks):
//   int4 header {segments, rows, entries, 0}; int2 next[8] (descriptors {offset, bytes}
//   of the following 8 chunks, {0, 0} past the end); int4 seg[segments] {first row,
//   rows, log2 lane-group size, 0}; int rows[pad4(r)]; int starts[pad4(r+1)];
//   int cols[pad4(e)]; T vals[e] (padded to 16 B); U only: T dinv[r] (padded).
__host__ __device__ __forceinline__ int pad4(int x) { return (x + 3) & ~3; }
__host__ __device__ __forceinline__ int pad16(int x) { return (x + 15) & ~15; }
__host__ __device__ __forceinline__ int chunk_bytes(int nseg, int r, int e, int tsz, bool upper) {
  return kChunkHdr + 16 * nseg + 4 * pad4(r) + 4 * pad4(r + 1) + 4 * pad4(e) + pad16(tsz * e) +
         (upper ? pad16(tsz * r) : 0);
}
// Grouped form (header .w = 1): int4 seg[segments]; int4 rowdesc[r] {output index, first
// entry, end entry, 0}; the entries: FP32 as (column bits, value) pairs of 8 bytes, FP64 as
// an int column array then a double value array (12 bytes an entry: the streams of many
// walkers share the L2).
__host__ __device__ __forceinline__ int chunk_bytes_grouped(int nseg, int r, int e, int tsz) {
  return kChunkHdr + 16 * nseg + 16 * r + (tsz == 4 ? pad16(8 * e) : pad16(4 * e) + pad16(8 * e));
}

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

// Exclusive prefix sum of a[0..cnt) in place (global or shared); returns the total.
__device__ __forceinline__ int block_scan_inplace(int* a, int cnt, Shared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int per = (cnt + nt - 1) / nt;
  const int b = min(cnt, tid * per), e = min(cnt, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += a[i];
  int inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) sh.redi[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? sh.redi[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += v;
    }
    if (lane < nw) sh.redi[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) sh.redi[32] = ti;
  }
  __syncthreads();
  int off = sh.redi[wid] + inc - s;
  for (int i = b; i < e; ++i) {
    const int t = a[i];
    a[i] = off;
    off += t;
  }
  const int total = sh.redi[32];
  __syncthreads();
  return total;
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
