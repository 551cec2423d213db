// vmc_krylov.cuh -- the per-move solve A_p z = e_r and the determinant ratio.
//
//   * M v = prod_s (I - z_hat_s u_s^T) Q (L U)^{-1} v                (Sec. 3.2 Eq. 18)
//     forward/backward substitution level by level (rows of a level in parallel),
//     then the column permutation Q, then the update chain fused into one pass:
//     c_s = u_s^T w_0 - sum_{t<s} G[s][t] c_t,  w = w_0 - sum_s z_hat_s c_s.
//   * right-preconditioned GMRES(m) on A_p M (Sec. 3.2 Eq. 15) with classical
//     Gram-Schmidt applied twice, Givens rotations, and the effective stability
//     N = max_j ||v_j - A_p M v_j||_2 over the Arnoldi vectors (Sec. 3.1 Eq. 10),
//     computed in the same pass as the first projections.
//   * FP64 iterative refinement: r = e_r - A_p x in FP64, inner GMRES in the working
//     precision T on r, x += d; the ratio 1 + u^T x (Sec. 3 Eq. 13) in FP64.
#pragma once
#include "vmc_precond.cuh"

namespace vmc {

template <typename T>
__device__ __forceinline__ const T* a_vals(const Walker& w);
template <>
__device__ __forceinline__ const float* a_vals<float>(const Walker& w) { return w.a_val32; }
template <>
__device__ __forceinline__ const double* a_vals<double>(const Walker& w) { return w.a_val; }

// 16-byte vector views of the Slater slots (slot starts are 16-byte aligned: cap % 4 == 0)
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  float v[4];
  __device__ __forceinline__ void load(const float* p) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  // streaming load (evict first): data read once per apply
  __device__ __forceinline__ void load_cs(const float* p) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct Vec4<double> {
  double v[4];
  __device__ __forceinline__ void load(const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ void load_cs(const double* p) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p + 2));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

// Dot product of Slater slot p (len entries, capacity cap) with x: 16-byte loads of
// four column indices and four values at a time (cap is a multiple of 4).  Up to 16
// entries at a time have their index and value loads issued together -- bounded by the
// slot's capacity, not its length, so the first ones need not wait for len -- then
// their gathers (entries < len only), then the products are summed in entry order.
template <typename T, typename X>
__device__ __forceinline__ X slot_dot(const int* __restrict__ cols, const T* __restrict__ vals, int len, int cap,
                                      const X* __restrict__ x) {
  constexpr int U = 4;
  X acc = 0;
  int q0 = 0;
  do {
    int4 c[U];
    Vec4<T> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = make_int4(0, 0, 0, 0);
      if (q0 + 4 * u < cap) {
        c[u] = *reinterpret_cast<const int4*>(cols + q0 + 4 * u);
        v[u].load(vals + q0 + 4 * u);
      }
    }
    X xv[4 * U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int q = q0 + 4 * u;
      xv[4 * u + 0] = q + 0 < len ? x[c[u].x] : (X)0;
      xv[4 * u + 1] = q + 1 < len ? x[c[u].y] : (X)0;
      xv[4 * u + 2] = q + 2 < len ? x[c[u].z] : (X)0;
      xv[4 * u + 3] = q + 3 < len ? x[c[u].w] : (X)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (q0 + 4 * u + k < len) acc += (X)v[u].v[k] * xv[4 * u + k];
    q0 += 4 * U;
  } while (q0 < len);
  return acc;
}

// y = A_p x: one particle's slot per thread, taken in slot order (consecutive threads
// read consecutive slots), the result scattered to the slot's row of A_p.  (Measured
// slower at n = 4096 x 256 walkers: two slots in flight per thread, 90 against 62 us; a
// warp staging 32 slots through shared memory with coalesced loads, 72 against 56 us.)
template <typename T>
__device__ __forceinline__ void spmv(const Walker& w, const Params& P, const T* __restrict__ x, T* __restrict__ y) {
  const T* av = a_vals<T>(w);
  const int n = w.n, cap = w.cap, nt = blockDim.x;
  for (int p = threadIdx.x; p < n; p += nt) {
    const int len = w.a_len[p], r = w.row_of_part[p];
    y[r] = slot_dot<T, T>(w.a_col + (size_t)p * cap, av + (size_t)p * cap, len, cap, x);
  }
}

// The SpMV's input vector, copied into the shared-memory solve-vector area when that
// holds one (idle between preconditioner applies): the SpMV's gathers then read shared
// memory instead of scattered global lines.  Block-wide; returns the vector to read.
template <typename T>
__device__ __forceinline__ const T* stage_x(const Walker& w, const Params& P, const T* x) {
  if (!P.y_smem) return x;
  T* xs = (T*)dyn_smem();
  __syncthreads();
  block_copy(xs, x, w.n);
  __syncthreads();
  return xs;
}

// Shared-memory ring of the stream chunks: one mbarrier per slot, initialised once
// per kernel launch; chunk g of the launch lives in slot g % S, phase (g / S) & 1.
__device__ __forceinline__ void ring_init(Shared& sh, const Params& P) {
  if (threadIdx.x == 0) {
    // a slot is released by every consumer warp once it is done with the chunk
    const unsigned rel = (unsigned)((blockDim.x >> 5) - 1);
    for (int s = 0; s < P.ring_slots; ++s) {
      mbar_init(&sh.bar[s], 1);
      mbar_init(&sh.ebar[s], rel);
    }
    sh.ring_seq = 0;
    sh.iflag[3] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// Entries of a grouped chunk (the layout of chunk_bytes_grouped): entry t is (column
// offset, value).
template <typename T>
struct GroupedEntries;
template <>
struct GroupedEntries<float> {
  const float2* p;
  __device__ __forceinline__ GroupedEntries(const unsigned char* ent, int) : p((const float2*)ent) {}
  __device__ __forceinline__ void get(int t, int& c, float& v) const {
    const float2 e = p[t];
    c = __float_as_int(e.x);
    v = e.y;
  }
};
template <>
struct GroupedEntries<double> {
  const int* c;
  const double* v;
  __device__ __forceinline__ GroupedEntries(const unsigned char* ent, int ne)
      : c((const int*)ent), v((const double*)(ent + pad16(4 * ne))) {}
  __device__ __forceinline__ void get(int t, int& cc, double& vv) const {
    cc = c[t];
    vv = v[t];
  }
};

// Producer of the chunk streams (lane 0 of the last warp): streams the factor's chunks
// into the ring with bulk copies, refilling a slot once the consumers have released it
// (the slot's "empty" barrier).  Returns the cycles spent waiting for free slots.
__device__ __forceinline__ long long stream_chunks(const unsigned char* stream, const int2* tab, int nch,
                                                   const Params& P, unsigned char* ring, int seq0, Shared& sh) {
  const int S = P.ring_slots;
  const int SB = P.slot_bytes;
  long long twait = 0;
  int2 pre[kMaxSlots];
  for (int k = 0; k < S && k < nch; ++k) pre[k] = tab[k];
  int slot = seq0 % S;
  int g = seq0;
  const unsigned long long pol = l2_policy_evict_last();
  for (int c = 0; c < nch; ++c, ++g) {
    unsigned char* dst = ring + (size_t)slot * SB;
    if (g >= S) {  // the consumers must have released the slot's previous use
      const long long tw = clock64();
      if (!mbar_wait(&sh.ebar[slot], (unsigned)(((g / S) - 1) & 1))) sh.iflag[3] = 1;
      twait += clock64() - tw;
    }
    // chunk c's descriptor: from the table for the first S chunks, else from the
    // header of chunk c - S, still in this slot
    const int2 tc = c < S ? pre[c] : ((const int2*)(dst + 16))[S - 1];
    mbar_expect_tx(&sh.bar[slot], (unsigned)tc.y);
    bulk_g2s_hint(dst, stream + tc.x, (unsigned)tc.y, &sh.bar[slot], pol);
    if (++slot == S) slot = 0;
  }
  return twait;
}

// One triangular solve in place on y (shared or global), level-synchronous.  The last
// warp produces (stream_chunks); the other warps solve: per chunk they wait for it to
// land, solve its segments (levels) one after the other with a barrier among the
// consumer warps between segments, and release the slot.  A segment marked for one
// warp (few rows) is solved by the first consumer warp alone, with only a warp
// synchronisation after it; the other consumer warps skip it and meet that warp at the
// barrier before the next segment solved by all.
// Lower: y_r -= sum_t L_rt y_t.  Upper: y_r = (y_r - sum_t U_rt y_t) / U_rr.
// Every wait gives up after ~1 s (status VMC_ERR_TIMEOUT).
template <typename T>
__device__ __forceinline__ void tri_staged(const Walker& w, const Params& P, bool upper, T* y, Shared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  const unsigned char* stream = upper ? w.ustream : w.lstream;
  const int2* tab = upper ? w.uchunk : w.lchunk;
  const int nch = upper ? w.ctl->nchunk_u : w.ctl->nchunk_l;
  const int S = P.ring_slots;
  const int SB = P.slot_bytes;
  unsigned char* ring = dyn_smem() + P.y_bytes;
  const int seq0 = sh.ring_seq;
  const int nct = nt - 32;
  long long twait = 0;
  if (wid == nwarp - 1) {
    if (lane == 0) twait = stream_chunks(stream, tab, nch, P, ring, seq0, sh);
  } else {
    int slot = seq0 % S;
    unsigned parity = (unsigned)((seq0 / S) & 1);
    long long tdata = 0;
    bool pend = false;  // the first warp solved rows the others have not synchronised with
    for (int c = 0; c < nch; ++c) {
      const long long tw0 = clock64();
      if (!mbar_wait(&sh.bar[slot], parity)) sh.iflag[3] = 1;
      tdata += clock64() - tw0;
      const unsigned char* ch = ring + (size_t)slot * SB;
      const int4 hd = *(const int4*)ch;
      const int nseg = hd.x, nr = hd.y, ne = hd.z;
      const int4* seg = (const int4*)(ch + kChunkHdr);
      const int* rws = (const int*)(ch + kChunkHdr + 16 * nseg);
      const int* st = rws + pad4(nr);
      const int* cl = st + pad4(nr + 1);
      const T* vl = (const T*)(cl + pad4(ne));
      const T* dv = (const T*)((const unsigned char*)vl + pad16((int)sizeof(T) * ne));
      if (hd.w) {
        // grouped form: the rows of a segment (group) are independent; each is a dot
        // product with the solution and input vectors at offsets from y (row descriptor
        // {output, first, end}; entries as (column, value) pairs)
        const int4* desc = (const int4*)(ch + kChunkHdr + 16 * nseg);
        const GroupedEntries<T> ent(ch + kChunkHdr + 16 * nseg + 16 * nr, ne);
        for (int sgi = 0; sgi < nseg; ++sgi) {
          const int4 sm = seg[sgi];
          const int r0 = sm.x, sr = sm.y, gs = sm.z;
          const int G = 1 << gs;
          const int gl = tid & (G - 1);
          const int ng = nct >> gs;
          for (int base = 0; base < sr; base += ng) {  // same trip count in every lane
            const int i = r0 + base + (tid >> gs);
            const bool on = base + (tid >> gs) < sr;
            T part = 0;
            int r = 0;
            if (on) {
              // expanded rows are long (up to exmax entries): FP32 keeps four entries in
              // flight per lane; FP64 two (every extra partial sum costs an FP64 add)
              const int4 d = desc[i];
              r = d.x;
              const int e = d.z;
              int t = d.y + gl;
              if constexpr (sizeof(T) == 4) {
                T p1 = 0, p2 = 0, p3 = 0;
                for (; t + 3 * G < e; t += 4 * G) {
                  int c0, c1, c2, c3;
                  T v0, v1, v2, v3;
                  ent.get(t, c0, v0);
                  ent.get(t + G, c1, v1);
                  ent.get(t + 2 * G, c2, v2);
                  ent.get(t + 3 * G, c3, v3);
                  part += v0 * y[c0];
                  p1 += v1 * y[c1];
                  p2 += v2 * y[c2];
                  p3 += v3 * y[c3];
                }
                for (; t < e; t += G) {
                  int c0;
                  T v0;
                  ent.get(t, c0, v0);
                  part += v0 * y[c0];
                }
                part = (part + p1) + (p2 + p3);
              } else {
                T p1 = 0;
                for (; t + G < e; t += 2 * G) {
                  int c0, c1;
                  T v0, v1;
                  ent.get(t, c0, v0);
                  ent.get(t + G, c1, v1);
                  part += v0 * y[c0];
                  p1 += v1 * y[c1];
                }
                if (t < e) {
                  int c0;
                  T v0;
                  ent.get(t, c0, v0);
                  part += v0 * y[c0];
                }
                part += p1;
              }
            }
            for (int o = G >> 1; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, G);
            if (on && gl == 0) y[r] = part;
          }
          asm volatile("bar.sync 1, %0;" ::"r"(nct) : "memory");  // group barrier (consumers)
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.ebar[slot]);
        if (++slot == S) { slot = 0; parity ^= 1u; }
        continue;
      }
      for (int sgi = 0; sgi < nseg; ++sgi) {
        const int4 sm = seg[sgi];
        const int r0 = sm.x, sr = sm.y;
        if (sm.w) {  // one warp
          if (wid == 0) {
            const int gs = sm.w - 1, G = 1 << gs, gl = lane & (G - 1);
            const int i = r0 + (lane >> gs);
            const bool on = (lane >> gs) < sr;
            T part = 0;
            int r = 0;
            if (on) {
              r = rws[i];
              T part2 = 0;
              const int e = st[i + 1];
              int t = st[i] + gl;
              for (; t + G < e; t += 2 * G) {
                part += vl[t] * y[cl[t]];
                part2 += vl[t + G] * y[cl[t + G]];
              }
              if (t < e) part += vl[t] * y[cl[t]];
              part += part2;
            }
            for (int o = G >> 1; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, G);
            if (on && gl == 0) {
              T acc = y[r] - part;
              if (upper) acc *= dv[i];
              y[r] = acc;
            }
            __syncwarp();
          }
          pend = true;
          continue;
        }
        if (pend) {  // publish the first warp's rows before a segment solved by all
          asm volatile("bar.sync 1, %0;" ::"r"(nct) : "memory");
          pend = false;
        }
        const int gs = sm.z;
        const int G = 1 << gs;
        const int gl = tid & (G - 1);
        const int ng = nct >> gs;
        for (int base = 0; base < sr; base += ng) {  // same trip count in every lane
          const int i = r0 + base + (tid >> gs);
          const bool on = base + (tid >> gs) < sr;
          T part = 0;
          int r = 0;
          if (on) {
            r = rws[i];
            T part2 = 0;
            const int e = st[i + 1];
            int t = st[i] + gl;
            for (; t + G < e; t += 2 * G) {  // two entries in flight per lane
              part += vl[t] * y[cl[t]];
              part2 += vl[t + G] * y[cl[t + G]];
            }
            if (t < e) part += vl[t] * y[cl[t]];
            part += part2;
          }
          for (int o = G >> 1; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, G);
          if (on && gl == 0) {
            T acc = y[r] - part;
            if (upper) acc *= dv[i];
            y[r] = acc;
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nct) : "memory");  // level barrier (consumers)
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.ebar[slot]);  // this warp is done with the chunk
      if (++slot == S) { slot = 0; parity ^= 1u; }
    }
    if (tid == 0) w.ctl->cyc[PH_TRIDATA] += tdata;
  }
  if (wid == nwarp - 1 && lane == 0) w.ctl->cyc[PH_TRIWAIT] += twait;
  __syncthreads();
  if (tid == 0) sh.ring_seq = seq0 + nch;
  __syncthreads();
}

// "Not yet solved" marker for the synchronisation-free solves: a quiet NaN with a
// payload that arithmetic never produces (GPU arithmetic returns the canonical NaN).
template <typename T>
struct Pending;
template <>
struct Pending<float> {
  static __device__ __forceinline__ float value() { return __int_as_float(0x7fc5a5a5); }
  static __device__ __forceinline__ bool is(float v) { return __float_as_int(v) == 0x7fc5a5a5; }
};
template <>
struct Pending<double> {
  static __device__ __forceinline__ double value() { return __longlong_as_double(0x7ff8a5a5a5a5a5a5ll); }
  static __device__ __forceinline__ bool is(double v) { return __double_as_longlong(v) == 0x7ff8a5a5a5a5a5a5ll; }
};
// Most retries of one row group's operands before giving up (status VMC_ERR_TIMEOUT).
constexpr int kSpinMax = 1 << 22;

// One triangular solve without level barriers: x = L^{-1} rhs (lower) or
// x = U^{-1} rhs (upper), x in shared memory pre-filled with Pending.  Rows are taken
// in the stream's level order, each by a group of G lanes (the level's group size),
// a warp's groups holding consecutive rows of one level.  A warp waits only until the
// operands of its own rows have been solved -- by whichever warp owns them -- instead
// of for the whole previous level; it retries as a unit, so its lanes stay converged.
// Rows only depend on earlier rows of the order, and every warp takes its rows in that
// order, so the waits always end.  Each row's sum is taken in the same order as the
// level-synchronous solve.
template <typename T>
__device__ __forceinline__ void tri_syncfree(const Walker& w, const Params& P, bool upper, const T* rhs, T* x,
                                             Shared& sh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarp = nt >> 5;
  const unsigned char* stream = upper ? w.ustream : w.lstream;
  const int2* tab = upper ? w.uchunk : w.lchunk;
  const int nch = upper ? w.ctl->nchunk_u : w.ctl->nchunk_l;
  const int S = P.ring_slots;
  const int SB = P.slot_bytes;
  unsigned char* ring = dyn_smem() + P.y_bytes;
  const int seq0 = sh.ring_seq;
  const int nct = nt - 32;
  const volatile T* xv = x;
  long long twait = 0;
  if (wid == nwarp - 1) {
    if (lane == 0) twait = stream_chunks(stream, tab, nch, P, ring, seq0, sh);
  } else {
    int slot = seq0 % S;
    unsigned parity = (unsigned)((seq0 / S) & 1);
    long long tdata = 0;
    for (int c = 0; c < nch; ++c) {
      const long long tw0 = clock64();
      if (!mbar_wait(&sh.bar[slot], parity)) sh.iflag[3] = 1;
      tdata += clock64() - tw0;
      const unsigned char* ch = ring + (size_t)slot * SB;
      const int4 hd = *(const int4*)ch;
      const int nseg = hd.x, nr = hd.y, ne = hd.z;
      const int4* seg = (const int4*)(ch + kChunkHdr);
      const int* rws = (const int*)(ch + kChunkHdr + 16 * nseg);
      const int* st = rws + pad4(nr);
      const int* cl = st + pad4(nr + 1);
      const T* vl = (const T*)(cl + pad4(ne));
      const T* dv = (const T*)((const unsigned char*)vl + pad16((int)sizeof(T) * ne));
      for (int sgi = 0; sgi < nseg; ++sgi) {
        const int4 sm = seg[sgi];
        const int r0 = sm.x, sr = sm.y, gs = sm.z;
        const int G = 1 << gs;
        const int gl = tid & (G - 1);
        const int ng = nct >> gs;
        for (int base = 0; base < sr; base += ng) {  // warp-uniform trip count
          const int i = base + (tid >> gs);
          const bool on = i < sr;
          int r = 0, t0 = 0, e = 0;
          if (on) {
            r = rws[r0 + i];
            t0 = st[r0 + i] + gl;
            e = st[r0 + i + 1];
          }
          // sum and readiness in one pass; the warp retries together until every lane's
          // operands were solved (so its lanes never diverge on a wait)
          T part = 0;
          for (int it = 0;; ++it) {
            T p1 = 0, p2 = 0;
            bool rdy = true;
            int t = t0;
            for (; t + G < e; t += 2 * G) {  // two entries in flight per lane
              const T a = xv[cl[t]], b = xv[cl[t + G]];
              rdy &= !Pending<T>::is(a) && !Pending<T>::is(b);
              p1 += vl[t] * a;
              p2 += vl[t + G] * b;
            }
            if (t < e) {
              const T a = xv[cl[t]];
              rdy &= !Pending<T>::is(a);
              p1 += vl[t] * a;
            }
            if (__all_sync(0xffffffffu, rdy)) { part = p1 + p2; break; }
            if (it >= kSpinMax || *(volatile int*)&sh.iflag[3]) { sh.iflag[3] = 1; break; }  // one give-up ends all waits
          }
          for (int o = G >> 1; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, G);
          if (on && gl == 0) {
            T acc = rhs[r] - part;
            if (upper) acc *= dv[r0 + i];
            ((volatile T*)x)[r] = acc;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.ebar[slot]);  // one arrival per consumer warp
      if (++slot == S) { slot = 0; parity ^= 1u; }
    }
    if (tid == 0) w.ctl->cyc[PH_TRIDATA] += tdata;
  }
  if (wid == nwarp - 1 && lane == 0) w.ctl->cyc[PH_TRIWAIT] += twait;
  __syncthreads();
  if (tid == 0) sh.ring_seq = seq0 + nch;
  __syncthreads();
}

// Both triangular solves on v (indexed by rows): returns the result L^{-1} then U^{-1}
// applied, in factor-label order (shared or global memory).  Block-wide.
template <typename T>
__device__ __forceinline__ const T* tri_both(const Walker& w, const Params& P, const T* v, Shared& sh) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x;
  T* y = P.y_smem ? (T*)dyn_smem() : (T*)w.tv;
  if (grouped_solves<T>(w, P)) {
    // two vectors [a | b]: v goes to b; L writes y_L into a reading b at offset +n; U
    // writes x into b (v is no longer needed) reading y_L at offset -n
    T* a = y;
    T* b = y + n;
    block_copy(b, v, n);
    __syncthreads();
    tri_staged<T>(w, P, false, a, sh);
    tri_staged<T>(w, P, true, b, sh);
    return b;
  }
  if (P.tri_sf) {
    T* x2 = (T*)(dyn_smem() + P.y_half);
    for (int i = tid; i < n; i += nt) { y[i] = Pending<T>::value(); x2[i] = Pending<T>::value(); }
    __syncthreads();
    tri_syncfree<T>(w, P, false, v, y, sh);
    tri_syncfree<T>(w, P, true, y, x2, sh);
    return x2;
  }
  block_copy(y, v, n);
  __syncthreads();
  tri_staged<T>(w, P, false, y, sh);
  tri_staged<T>(w, P, true, y, sh);
  return y;
}

// z = M v  (v indexed by rows, z by columns of A_p).  Block-wide, ends synchronised.
template <typename T>
__device__ __noinline__ void precond_apply(const Walker& w, const Params& P, const T* __restrict__ v,
                                           T* __restrict__ z, Shared& sh) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x;
  const long long t0 = clock64();
  const T* y = tri_both<T>(w, P, v, sh);
  const long long t1 = clock64();
  if (tid == 0) {
    Ctl* c = w.ctl;
    c->cyc[PH_TRI] += t1 - t0;
    // factor values + indices, diagonal, v read, z write, the level-row records
    c->alg_bytes += c->nnz_LU * (sizeof(T) + 4) + (double)n * (3 * sizeof(T) + 8);
  }
  block_scatter(z, w.perm, y, n);
  __syncthreads();
  const int mu = w.ctl->n_upd;
  if (mu > 0) {
    const T* Zt = (const T*)w.upd_z;  // z_hat stored transposed: Zt[i * mu_cap + s]
    const int mcap = w.mu4;
    const T* Uv = (const T*)w.upd_uval;
    const int lane = tid & 31, wid = tid >> 5;
    // d_s = u_s^T w_0 for all s at once: a lane group per update
    int gs = 0;
    while (gs < 5 && (mu << (gs + 1)) <= nt) ++gs;
    const int G = 1 << gs, gl = tid & (G - 1);
    for (int base = 0; base < mu; base += (nt >> gs)) {
      const int s_ = base + (tid >> gs);
      double acc = 0.0;
      if (s_ < mu) {
        const int ul = w.upd_ulen[s_];
        const int* uc = w.upd_ucol + (size_t)s_ * kMaxU;
        const T* uu = Uv + (size_t)s_ * kMaxU;
        for (int t = gl; t < ul; t += G) acc += (double)uu[t] * (double)z[uc[t]];
      }
      for (int o = G >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
      if (s_ < mu && gl == 0) sh.cupd[s_] = acc;
    }
    // G[t][s] (t > s) for the substitution, staged in the idle stream ring when it fits
    // (the ring's last writer was the bulk-copy proxy: order the generic stores after it)
    double* Gs = nullptr;
    if ((size_t)mu * mu * sizeof(double) <= (size_t)P.ring_slots * P.slot_bytes) {
      Gs = reinterpret_cast<double*>(dyn_smem() + P.y_bytes);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int idx = tid; idx < mu * mu; idx += nt) {
        const int t = idx / mu, s2 = idx - t * mu;
        Gs[idx] = s2 < t ? w.upd_G[(size_t)t * kMaxUpd + s2] : 0.0;
      }
    }
    __syncthreads();
    // c_s = d_s - sum_{t<s} G[s][t] c_t: warp 0, lane t holds d_t for t = lane + 32 k;
    // each solved c_s is broadcast and subtracted from the later d_t
    if (wid == 0) {
      double d[kMaxUpd / 32];
#pragma unroll
      for (int k = 0; k < kMaxUpd / 32; ++k) d[k] = lane + 32 * k < mu ? sh.cupd[lane + 32 * k] : 0.0;
      for (int s_ = 0; s_ < mu; ++s_) {
        const double cs = __shfl_sync(0xffffffffu, d[s_ >> 5], s_ & 31);
#pragma unroll
        for (int k = 0; k < kMaxUpd / 32; ++k) {
          const int t = lane + 32 * k;
          if (t > s_ && t < mu) d[k] -= (Gs ? Gs[t * mu + s_] : w.upd_G[(size_t)t * kMaxUpd + s_]) * cs;
        }
      }
#pragma unroll
      for (int k = 0; k < kMaxUpd / 32; ++k)
        if (lane + 32 * k < mu) sh.cupd[lane + 32 * k] = d[k];
    }
    if (Gs) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // before the ring's next bulk copies
    __syncthreads();
    // w = w_0 - sum_s z_hat_s c_s: row i of Zt is contiguous over s (streaming loads: the
    // chain is read once per apply and should not push the chunk streams out of L2)
    for (int i = tid; i < n; i += nt) {
      const T* zr = Zt + (size_t)i * mcap;
      T acc = z[i];
      int s_ = 0;
      for (; s_ + 4 <= mu; s_ += 4) {
        Vec4<T> v;
        v.load_cs(zr + s_);
        acc -= v.v[0] * (T)sh.cupd[s_] + v.v[1] * (T)sh.cupd[s_ + 1] + v.v[2] * (T)sh.cupd[s_ + 2] +
               v.v[3] * (T)sh.cupd[s_ + 3];
      }
      for (; s_ < mu; ++s_) acc -= zr[s_] * (T)sh.cupd[s_];
      z[i] = acc;
    }
    __syncthreads();
  }
  if (tid == 0) {
    Ctl* c = w.ctl;
    c->cyc[PH_CHAIN] += clock64() - t1;
    // z_hat vectors, sparse u vectors, z read + write
    if (mu > 0) c->alg_bytes += (double)mu * n * sizeof(T) + (double)c->upd_nnz * (sizeof(T) + 4) + 2.0 * n * sizeof(T);
  }
}

// Dot products <V_k, wv> for k = 0..nk-1 into out[k]; if mon, also ||V_{nk-1} - wv||^2
// into out[nk] and ||wv||^2 into out[nk + 1].  One warp per dot.  Ends synchronised.
template <typename T>
__device__ __forceinline__ void multi_dot(const T* __restrict__ V, int n, int nk, const T* __restrict__ wv,
                                          double* out, bool mon) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int total = nk + (mon ? 2 : 0);
  for (int k = wid; k < total; k += nw) {
    T a0 = 0, a1 = 0;
    if (k < nk) {
      const T* vk = V + (size_t)k * n;
      int i = lane;
      for (; i + 32 < n; i += 64) { a0 += vk[i] * wv[i]; a1 += vk[i + 32] * wv[i + 32]; }
      if (i < n) a0 += vk[i] * wv[i];
    } else if (k == nk) {
      const T* vk = V + (size_t)(nk - 1) * n;
      for (int i = lane; i < n; i += 32) { const T d = vk[i] - wv[i]; a0 += d * d; }
    } else {
      for (int i = lane; i < n; i += 32) a0 += wv[i] * wv[i];
    }
    const double s = warp_sum((double)a0 + (double)a1);
    if (lane == 0) out[k] = s;
  }
  __syncthreads();
}

// Right-preconditioned GMRES(m) on A_p M d = rhs (FP64 rhs, norm beta); adds the
// correction M V y into x64.  Returns the iteration count; conv (reached rtol), the
// monitor N and, when its_trig is given, the iteration at which the residual estimate
// first reached trig * beta (-1: not in this cycle; the controller's convergence test).
template <typename T>
__device__ __noinline__ int gmres_inner(const Walker& w, const Params& P, double beta, double rtol, bool& conv,
                           double& Nmon, Shared& sh, double trig = 0.0, int* its_trig = nullptr) {
  const int n = w.n, tid = threadIdx.x, nt = blockDim.x, m = P.m;
  T* V = (T*)w.V;
  T* Zk = (T*)w.Zk;
  const double inv = 1.0 / beta;
  for (int i = tid; i < n; i += nt) V[i] = (T)(w.r64[i] * inv);
  if (tid == 0) { sh.g[0] = beta; sh.iflag[1] = 0; sh.iflag[8] = -1; }
  double mon2 = 0.0;
  __syncthreads();
  int j = 0;
  for (; j < m;) {
    T* vj = V + (size_t)j * n;
    T* zj = Zk + (size_t)j * n;
    T* wv = V + (size_t)(j + 1) * n;
    precond_apply<T>(w, P, vj, zj, sh);
    const long long ts = clock64();
    spmv<T>(w, P, stage_x<T>(w, P, zj), wv);
    __syncthreads();
    const long long to = clock64();
    if (tid == 0) {
      Ctl* c = w.ctl;
      c->cyc[PH_SPMV] += to - ts;
      // SpMV: values + indices, x read, y write; the first Gram-Schmidt pass: projections
      // (V_0..V_j and w read) and update (V_0..V_j and w read, w written), normalisation
      c->alg_bytes += c->nnz_A * (sizeof(T) + 4) + (double)n * (2 * sizeof(T) + 4) +
                      (double)n * sizeof(T) * (2.0 * (j + 1) + 6.0);
    }
    multi_dot<T>(V, n, j + 1, wv, sh.h1, true);          // projections, monitor, ||w||^2
    mon2 = fmax(mon2, sh.h1[j + 1]);
    const double w2 = sh.h1[j + 2];
    T nrm_t = 0;
    for (int i = tid; i < n; i += nt) {
      T acc = wv[i];
      for (int k = 0; k <= j; ++k) acc -= (T)sh.h1[k] * V[(size_t)k * n + i];
      wv[i] = acc;
      nrm_t += acc * acc;
    }
    double nrm2 = block_sum((double)nrm_t, sh);
    // second Gram-Schmidt pass only when the first cancelled much of w: ||w'|| < ||w|| / sqrt(2)
    // (Daniel, Gragg, Kaufman, Stewart 1976); else its coefficients are taken as zero
    if (2.0 * nrm2 < w2) {
      if (tid == 0) w.ctl->alg_bytes += (double)n * sizeof(T) * (2.0 * (j + 1) + 3.0);  // the second pass
      multi_dot<T>(V, n, j + 1, wv, sh.h2, false);
      nrm_t = 0;
      for (int i = tid; i < n; i += nt) {
        T acc = wv[i];
        for (int k = 0; k <= j; ++k) acc -= (T)sh.h2[k] * V[(size_t)k * n + i];
        wv[i] = acc;
        nrm_t += acc * acc;
      }
      nrm2 = block_sum((double)nrm_t, sh);
    } else {
      if (tid <= j) sh.h2[tid] = 0.0;
      __syncthreads();
    }
    const double nrm = sqrt(nrm2);
    const T sc = nrm > 0.0 ? (T)(1.0 / nrm) : (T)0;
    for (int i = tid; i < n; i += nt) wv[i] *= sc;
    if (tid == 0) {
      double* H = sh.H;
      for (int k = 0; k <= j; ++k) H[k * kMaxM + j] = sh.h1[k] + sh.h2[k];
      H[(j + 1) * kMaxM + j] = nrm;
      for (int k = 0; k < j; ++k) {
        const double a0 = H[k * kMaxM + j], a1 = H[(k + 1) * kMaxM + j];
        H[k * kMaxM + j] = sh.cs[k] * a0 + sh.sn[k] * a1;
        H[(k + 1) * kMaxM + j] = -sh.sn[k] * a0 + sh.cs[k] * a1;
      }
      const double a0 = H[j * kMaxM + j], a1 = H[(j + 1) * kMaxM + j];
      const double rr = sqrt(a0 * a0 + a1 * a1);
      sh.cs[j] = rr == 0.0 ? 1.0 : a0 / rr;
      sh.sn[j] = rr == 0.0 ? 0.0 : a1 / rr;
      H[j * kMaxM + j] = rr;
      H[(j + 1) * kMaxM + j] = 0.0;
      sh.g[j + 1] = -sh.sn[j] * sh.g[j];
      sh.g[j] = sh.cs[j] * sh.g[j];
      sh.iflag[1] = (fabs(sh.g[j + 1]) <= rtol * beta) || nrm == 0.0;
      if (sh.iflag[8] < 0 && fabs(sh.g[j + 1]) <= trig * beta) sh.iflag[8] = j + 1;
      w.ctl->cyc[PH_ORTH] += clock64() - to;
    }
    __syncthreads();
    ++j;
    if (sh.iflag[1]) break;
  }
  conv = sh.iflag[1] != 0;
  if (its_trig) *its_trig = sh.iflag[8];
  Nmon = sqrt(mon2);
  if (tid == 0) {
    const double* H = sh.H;
    for (int k = j - 1; k >= 0; --k) {
      double acc = sh.g[k];
      for (int l = k + 1; l < j; ++l) acc -= H[k * kMaxM + l] * sh.y[l];
      sh.y[k] = H[k * kMaxM + k] != 0.0 ? acc / H[k * kMaxM + k] : 0.0;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    T acc = 0;
    for (int k = 0; k < j; ++k) acc += (T)sh.y[k] * Zk[(size_t)k * n + i];
    w.x64[i] += (double)acc;
  }
  if (tid == 0) w.ctl->alg_bytes += (double)n * (j * sizeof(T) + 16.0);  // Zk y, x read + write
  __syncthreads();
  return j;
}

// r64 = e_brow - A_p x64 (FP64); returns ||r64||_2 and, in *xnorm, ||x64||_2.
// Ends synchronised.
__device__ __forceinline__ double residual64(const Walker& w, int brow, double* xnorm, Shared& sh) {
  const int n = w.n, cap = w.cap, nt = blockDim.x;
  const long long t0 = clock64();
  double ss = 0.0, xx = 0.0;
  for (int p = threadIdx.x; p < n; p += nt) {  // slots in order (see spmv)
    const int len = w.a_len[p], r = w.row_of_part[p];
    const double acc = slot_dot<double, double>(w.a_col + (size_t)p * cap, w.a_val + (size_t)p * cap, len, cap, w.x64);
    const double rr = (r == brow ? 1.0 : 0.0) - acc;
    w.r64[r] = rr;
    ss += rr * rr;
    const double xp = w.x64[p];
    xx += xp * xp;
  }
  *xnorm = sqrt(block_sum(xx, sh));
  const double rn = sqrt(block_sum(ss, sh));
  if (threadIdx.x == 0) {
    Ctl* c = w.ctl;
    c->cyc[PH_RESID] += clock64() - t0;
    c->alg_bytes += c->nnz_A * 12.0 + (double)n * 24.0;  // FP64 A, x read, r write, row lengths
  }
  return rn;
}

// u^T x64 over the u list in shared memory (FP64).
__device__ __forceinline__ double u_dot_x(const Walker& w, Shared& sh) {
  double acc = 0.0;
  for (int t = threadIdx.x; t < sh.ulen; t += blockDim.x) acc += sh.uval[t] * w.x64[sh.ucol[t]];
  return block_sum(acc, sh);
}

struct SolveOut {
  double ratio;
  int its1;          // iterations of the first cycle
  bool conv1;        // the first cycle reached its tolerance
  int its_trig;      // iterations (all cycles) until the residual reached Params::trig_rtol; -1: never
  double N;
  int passes;
  int total_its;
  int status;
};

// First pass from x = 0 (used by the controller), then refinement passes until the
// predicted ratio error |u^T d| ||r_j|| / ||r_{j-1}|| <= ratio_tol max(|ratio|, 1e-3).
template <typename T>
__device__ void solve_first(const Walker& w, const Params& P, int brow, double rtol, SolveOut& o, Shared& sh) {
  const int n = w.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    w.x64[i] = 0.0;
    w.r64[i] = i == brow ? 1.0 : 0.0;
  }
  __syncthreads();
  bool conv = false;
  double N = 0.0;
  int at = -1;
  o.its1 = gmres_inner<T>(w, P, 1.0, rtol, conv, N, sh, P.trig_rtol, &at);
  o.conv1 = conv;
  o.its_trig = at;
  o.N = N;
  o.total_its = o.its1;
  o.passes = 1;
}

// Refinement: the ratio error after a pass is u^T A^{-1} r.  It is predicted as the
// larger of |u^T d_j| ||r_j|| / ||r_{j-1}|| (the last correction scaled by the last
// residual reduction) and ||u|| ||x|| ||r_j|| (||x|| ~ ||A^{-1} e_r|| as a norm
// estimate), and passes continue until it is <= ratio_tol max(|ratio|, 1e-3).  Each
// pass asks the inner GMRES for only the reduction the goal needs (never below
// rtol_floor).
template <typename T>
__device__ __noinline__ void refine(const Walker& w, const Params& P, int brow, double rtol_floor, int max_passes, SolveOut& o,
                       Shared& sh) {
  double usq = 0.0;
  for (int t = threadIdx.x; t < sh.ulen; t += blockDim.x) usq += sh.uval[t] * sh.uval[t];
  const double unorm = sqrt(block_sum(usq, sh));
  double ratio_prev = 1.0;
  double rprev = 1.0;
  double ratio = 1.0 + u_dot_x(w, sh);
  double xn = 0.0;
  double rn = residual64(w, brow, &xn, sh);
  o.status = ST_OK;
  for (;;) {
    // ||e_r|| = 1: the FP64 residual norm is also the relative residual
    if (o.its_trig < 0 && rn <= P.trig_rtol) o.its_trig = o.total_its;
    const double delta = fabs(ratio - ratio_prev);
    const double pred = fmax(delta * rn / rprev, unorm * xn * rn);
    const double goal = P.ratio_tol * fmax(fabs(ratio), 1e-3);
    if (pred <= goal || rn == 0.0) break;
    if (o.passes >= max_passes) {
      if (rn > 1e-6) o.status = ST_NOCONV;
      break;
    }
    double need = 0.1 * goal / pred;
    need = fmin(fmax(need, rtol_floor), 0.1);
    bool conv = false;
    double N = 0.0;
    int at = -1;
    const int its = gmres_inner<T>(w, P, rn, need, conv, N, sh, P.trig_rtol / rn, &at);
    if (o.its_trig < 0 && at > 0) o.its_trig = o.total_its + at;
    o.total_its += its;
    o.passes += 1;
    ratio_prev = ratio;
    rprev = rn;
    ratio = 1.0 + u_dot_x(w, sh);
    rn = residual64(w, brow, &xn, sh);
  }
  o.ratio = ratio;
}

}  // namespace vmc
