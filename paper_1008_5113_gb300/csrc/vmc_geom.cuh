// vmc_geom.cuh -- device RNG, proposals and the Slater-row builder.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of
// two 32x32->64-bit products; the key bumped by the Weyl constants between rounds),
// keyed by the walker's 64-bit seed with counter (sweep, particle, purpose, j);
// purposes: 0 initial jitter, 1 proposal, 2 Metropolis uniform.  Normals by
// Box-Muller; uniforms u = (top 52 bits + 1/2) 2^-52, strictly inside (0, 1).
//
// Geometry arithmetic uses explicitly rounded FP64 operations (no FMA contraction)
// so that positions, minimum-image distances and the cutoff test d^2 <= r_c^2 are
// the plainly rounded IEEE results.
#pragma once
#include "vmc_device.cuh"

namespace vmc {

__host__ __device__ __forceinline__ void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u01(uint32_t hi, uint32_t lo) {
  const uint64_t x = (((uint64_t)hi << 32) | lo) >> 12;
  return __dmul_rn((double)x + 0.5, 1.0 / 4503599627370496.0);
}

__device__ __forceinline__ void draw(uint64_t seed, uint32_t sweep, uint32_t particle, uint32_t purpose,
                                     uint32_t j, uint32_t out[4]) {
  const uint32_t ctr[4] = {sweep, particle, purpose, j};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox4x32_10(ctr, key, out);
}

__device__ __forceinline__ void normal3(uint64_t seed, uint32_t sweep, uint32_t particle, uint32_t purpose,
                                        double z[3]) {
  const double two_pi = 6.283185307179586;  // 2 pi rounded to FP64
  uint32_t wv[4];
  draw(seed, sweep, particle, purpose, 0u, wv);
  double rad = sqrt(__dmul_rn(-2.0, log(u01(wv[0], wv[1]))));
  double s, c;
  sincos(__dmul_rn(two_pi, u01(wv[2], wv[3])), &s, &c);
  z[0] = __dmul_rn(rad, c);
  z[1] = __dmul_rn(rad, s);
  draw(seed, sweep, particle, purpose, 1u, wv);
  rad = sqrt(__dmul_rn(-2.0, log(u01(wv[0], wv[1]))));
  z[2] = __dmul_rn(rad, cos(__dmul_rn(two_pi, u01(wv[2], wv[3]))));
}

__device__ __forceinline__ double accept_uniform(uint64_t seed, uint32_t sweep, uint32_t particle) {
  uint32_t wv[4];
  draw(seed, sweep, particle, 2u, 0u, wv);
  return u01(wv[0], wv[1]);
}

// wrap into [0, L)
__device__ __forceinline__ double wrap_box(double x, double L) {
  double y = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
  if (y >= L) y = __dsub_rn(y, L);
  return y;
}
__device__ __forceinline__ double min_image(double d, double L) {
  return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}
__device__ __forceinline__ double dist2(const double* r, const double* z, double L) {
  const double dx = min_image(__dsub_rn(r[0], z[0]), L);
  const double dy = min_image(__dsub_rn(r[1], z[1]), L);
  const double dz = min_image(__dsub_rn(r[2], z[2]), L);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Candidate cells around r: per axis the cells floor((r-rc)/a)-1 .. floor((r+rc)/a)+1,
// at most K of them (a full period).  Candidate q enumerates (basis fastest, then x, y, z).
struct CandBox {
  int lo[3], cnt[3];
  int total;
};
__device__ __forceinline__ CandBox cand_box(const Walker& w, const double* r) {
  CandBox b;
  for (int d = 0; d < 3; ++d) {
    const int lo = (int)floor((r[d] - w.rc) / w.a) - 1;
    const int hi = (int)floor((r[d] + w.rc) / w.a) + 1;
    b.lo[d] = lo;
    b.cnt[d] = min(hi - lo + 1, w.K);
  }
  b.total = b.cnt[0] * b.cnt[1] * b.cnt[2] * w.per;
  return b;
}
__device__ __forceinline__ int cand_site(const Walker& w, const CandBox& b, int q) {
  const int bb = q % w.per;
  int t = q / w.per;
  const int ix = t % b.cnt[0];
  t /= b.cnt[0];
  const int iy = t % b.cnt[1];
  const int iz = t / b.cnt[1];
  const int K = w.K;
  const int cx = ((b.lo[0] + ix) % K + K) % K;
  const int cy = ((b.lo[1] + iy) % K + K) % K;
  const int cz = ((b.lo[2] + iz) % K + K) % K;
  return (cx + K * (cy + K * cz)) * w.per + bb;
}

// One warp builds the Slater row of a particle at r (Sec. 2.1 Eq. 3): the columns
// (positions of the orbitals) and values exp(-kappa d^2) for every orbital with
// min-image d^2 <= r_c^2, in candidate order.  Returns the count, or -1 if the row
// exceeds cap (callers turn that into ST_CAPACITY).
__device__ __forceinline__ int build_row_warp(const Walker& w, const double* r, int* ocol, double* oval,
                                              int cap) {
  const int lane = threadIdx.x & 31;
  const CandBox b = cand_box(w, r);
  int cnt = 0;
  for (int base = 0; base < b.total; base += 32) {
    const int q = base + lane;
    bool keep = false;
    double v = 0.0;
    int col = 0;
    if (q < b.total) {
      const int j = cand_site(w, b, q);
      const double d2 = dist2(r, w.Z + 3 * j, w.L);
      if (d2 <= w.rc2) {
        keep = true;
        v = exp(__dmul_rn(-w.kappa, d2));
        col = w.col_of_orb[j];
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int slot = cnt + __popc(m & lanemask_lt());
    if (keep && slot < cap) { ocol[slot] = col; oval[slot] = v; }
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt > cap ? -1 : cnt;
}

// One warp forms u = a' - a_p (Sec. 3 Eq. 12) from the new row (acol/aval, alen) and
// the stored row of particle p; output in ucol/uval (entries of a' first, then the
// entries of a_p that a' lacks).  Returns the count.
__device__ __forceinline__ int build_u_warp(const Walker& w, int p, const int* acol, const double* aval,
                                            int alen, int* ucol, double* uval) {
  const int lane = threadIdx.x & 31;
  const int olen = w.a_len[p];
  const int* oc = w.a_col + (size_t)p * w.cap;
  const double* ov = w.a_val + (size_t)p * w.cap;
  int cnt = 0;
  for (int base = 0; base < alen; base += 32) {
    const int t = base + lane;
    double v = 0.0;
    int c = 0;
    if (t < alen) {
      c = acol[t];
      v = aval[t];
      for (int s = 0; s < olen; ++s)
        if (oc[s] == c) { v = __dsub_rn(v, ov[s]); break; }
    }
    const unsigned m = __ballot_sync(0xffffffffu, t < alen);
    if (t < alen) { ucol[cnt + t - base] = c; uval[cnt + t - base] = v; }
    cnt += __popc(m);
  }
  for (int base = 0; base < olen; base += 32) {
    const int t = base + lane;
    bool extra = false;
    int c = 0;
    double v = 0.0;
    if (t < olen) {
      c = oc[t];
      extra = true;
      for (int s = 0; s < alen; ++s)
        if (acol[s] == c) { extra = false; break; }
      v = -ov[t];
    }
    const unsigned m = __ballot_sync(0xffffffffu, extra);
    const int slot = cnt + __popc(m & lanemask_lt());
    if (extra) { ucol[slot] = c; uval[slot] = v; }
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

}  // namespace vmc
