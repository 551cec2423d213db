// vmc_capi.cu -- the C ABI (include/vmc.h): context, device memory, launches,
// host-side geometry/layout, statistics and inspection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vmc.h"
#include "vmc_internal.h"

using namespace vmc;

// ---------------------------------------------------------------------------
// layout: sites (Sec. 2.1, Sec. 4), the fixed colour order of orbitals, and a
// rigorous bound on the number of orbitals within r_c of any point.
// ---------------------------------------------------------------------------
namespace vmc {

int expanded_row_cap(int capLU, int row_cap) {
  const int c = row_cap > 0 ? row_cap : std::min(2 * capLU, 160);
  return (std::max(capLU + 4, c) + 3) / 4 * 4;
}

// One factor row of either stream form (FP64, with its diagonal) fits the smallest ring slot.
bool rows_fit_slot(int cap, int lfil_extra, int row_cap) {
  const int pmax = lfil_extra >= 0 ? lfil_extra : (cap + 1) / 2;
  const int capLU = (cap + pmax + 2 + 3) / 4 * 4;
  const int mx = std::max(capLU, expanded_row_cap(capLU, row_cap));
  return chunk_bytes(1, 1, mx, 8, true) <= kSlotBytes && chunk_bytes_grouped(1, 1, mx, 8) <= kSlotBytes;
}

void plan_smem(int ybytes, int budget, Params& P, bool allow_sf) {
  int avail = budget;
  P.tri_sf = 0;
  P.y_half = 0;
  if (allow_sf && 2 * ybytes + 4 * kSlotBytes <= budget) {
    P.tri_sf = 1;  // both solve vectors in shared memory: synchronisation-free solves
    P.y_smem = 1;
    P.y_bytes = 2 * ybytes;
    P.y_half = ybytes;
    avail = budget - 2 * ybytes;
  } else if (ybytes + 2 * kSlotBytes <= budget) {
    P.y_smem = 1;
    P.y_bytes = ybytes;
    avail = budget - ybytes;
  } else {
    P.y_smem = 0;
    P.y_bytes = 0;
  }
  P.slot_bytes = avail >= 4 * 2 * kSlotBytes ? 2 * kSlotBytes : kSlotBytes;
  P.ring_slots = std::min(kMaxSlots, avail / P.slot_bytes);
  // the rest of the budget is ILUTP scratch (work row, U-row cache)
  P.dsm_bytes = std::max(budget, P.y_bytes + P.ring_slots * P.slot_bytes);
}

static int count_sites_within(int lattice, double a, double gx, double gy, double gz, double R) {
  const int per = lattice == 1 ? 2 : 1;
  int cnt = 0;
  const int lo[3] = {(int)std::floor((gx - R) / a) - 1, (int)std::floor((gy - R) / a) - 1, (int)std::floor((gz - R) / a) - 1};
  const int hi[3] = {(int)std::floor((gx + R) / a) + 1, (int)std::floor((gy + R) / a) + 1, (int)std::floor((gz + R) / a) + 1};
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x)
        for (int b = 0; b < per; ++b) {
          const double off = 0.5 * b;
          const double dx = gx - a * (x + off), dy = gy - a * (y + off), dz = gz - a * (z + off);
          if (dx * dx + dy * dy + dz * dz <= R * R) ++cnt;
        }
  return cnt;
}

int make_layout(int K, int lattice, double a, double r_c, Layout& out, const char** why) {
  if (K < 2 || K > 64) { *why = "K must be in [2, 64]"; return 1; }
  if (lattice != 0 && lattice != 1) { *why = "lattice must be 0 (sc) or 1 (bcc)"; return 1; }
  if (!(a > 0.0) || !(r_c > 0.0)) { *why = "a and r_c must be positive"; return 1; }
  const double L = K * a;
  if (!(r_c < 0.5 * L)) { *why = "r_c must be below half the box side"; return 1; }
  const double cover = lattice == 1 ? a * std::sqrt(5.0) / 4.0 : a * std::sqrt(3.0) / 2.0;
  if (!(r_c > cover)) { *why = "r_c must exceed the lattice covering radius (else A can be singular)"; return 1; }
  const int per = lattice == 1 ? 2 : 1;
  const int n = K * K * K * per;
  out.n = n;
  out.per = per;
  out.Z.assign((size_t)n * 3, 0.0);
  for (int jz = 0; jz < K; ++jz)
    for (int jy = 0; jy < K; ++jy)
      for (int jx = 0; jx < K; ++jx)
        for (int b = 0; b < per; ++b) {
          const int j = (jx + K * (jy + K * jz)) * per + b;
          const double off = 0.5 * (double)b;
          out.Z[3 * j + 0] = a * ((double)jx + off);
          out.Z[3 * j + 1] = a * ((double)jy + off);
          out.Z[3 * j + 2] = a * ((double)jz + off);
        }
  // colour of orbital j: (x mod 3, y mod 3, z mod 3, basis); same-colour sites are >= 3a
  // apart (except across the periodic seam when 3 does not divide K)
  std::vector<std::pair<int, int>> key(n);
  for (int j = 0; j < n; ++j) {
    const int cell = j / per, b = j % per;
    const int cx = cell % K, cy = (cell / K) % K, cz = cell / (K * K);
    key[j] = {(cx % 3) + 3 * (cy % 3) + 9 * (cz % 3) + 27 * b, j};
  }
  std::sort(key.begin(), key.end());
  out.orb_of_col.assign(n, 0);
  out.col_of_orb.assign(n, 0);
  for (int c = 0; c < n; ++c) {
    out.orb_of_col[c] = key[c].second;
    out.col_of_orb[key[c].second] = c;
  }
  // Row capacity: every point lies within h sqrt(3)/2 of a grid point g (spacing h),
  // so count(point, r_c) <= count(g, r_c + h sqrt(3)/2); the lattice has period a.
  const int G = 16;
  const double h = a / G, R = r_c + h * std::sqrt(3.0) / 2.0;
  int mx = 0;
  for (int z = 0; z <= G; ++z)
    for (int y = 0; y <= G; ++y)
      for (int x = 0; x <= G; ++x) mx = std::max(mx, count_sites_within(lattice, a, x * h, y * h, z * h, R));
  out.cap = (std::min(n, mx) + 3) / 4 * 4;  // multiple of 4: 16-byte slot loads stay in the slot
  if (out.cap > kMaxRow) { *why = "r_c too large: a Slater row could exceed 256 orbitals"; return 1; }
  return 0;
}

}  // namespace vmc

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct vmc_ctx {
  int nw = 0;
  std::vector<vmc_system> sys;
  vmc_solver_params prm{};
  Params P{};
  cudaStream_t stream = nullptr;
  int threads = 256;
  int row_cap = 0;  // trisolve_row_cap
  bool fp64 = false;
  std::vector<Walker> hw;
  Walker* dW = nullptr;
  Ctl* dCtl = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  size_t smem = 0;
  int64_t sweeps = 0;
  std::string err;
  long long total_n = 0;
  int max_n = 0;
  uint64_t* d_seeds = nullptr;
  uint8_t* d_acc = nullptr;
  double* d_ratio = nullptr;
  size_t log_cap = 0;
  std::vector<char> pending;
  bool ready = false;
  bool dense = false;
  // background refactorisation: second factor set views, factor-CTA views, launch ids
  bool pair = false;
  std::vector<Walker> hw1, hwf;
  Walker* dW1 = nullptr;
  Walker* dWf = nullptr;
  Ctl* dShadow = nullptr;
  int launch_seq = 0;
  double* d_energy = nullptr;  // kinetic energies, one per walker (in the arena)
  unsigned long long* d_budget = nullptr;  // move counter of the budgeted advance (in the arena)
  // CUDA graph of one sweep of the STEP / PLAIN engines (replayed once per sweep)
  cudaGraphExec_t graph = nullptr;
  cudaStream_t capture_stream = nullptr;
  long long* d_sweep = nullptr;
  const void* g_seeds = nullptr;
  const void* g_acc = nullptr;
  const void* g_ratio = nullptr;
  double g_sigma = 0.0;
  int g_limit = -1;
};

static vmc_status fail(vmc_ctx* c, vmc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}
static vmc_status cuda_fail(vmc_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? VMC_ERR_OOM : VMC_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}
#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

static LaunchCfg cfg(const vmc_ctx* c) { return LaunchCfg{c->stream, c->threads, c->fp64, c->smem}; }

// Automatic background refactorisation (refactor_lag = -1) needs every walker pair on
// the GPU at once, and systems small enough that a factorisation by one warp finishes
// within the accepts between adoptions: at n = 1000 it takes a fraction of them, at
// n = 32768 (about 28 s) many times more, and in-line refactoring is faster there.
constexpr long long kAutoPairMaxN = 8192;

static bool auto_pairs_fit(const vmc_system* systems, int n_walkers, int nsm) {
  if (nsm <= 0 || 2 * n_walkers > nsm) return false;
  for (int w = 0; w < n_walkers; ++w) {
    const long long K = std::min(std::max(systems[w].K, 0), 1 << 10);
    if (K * K * K * (systems[w].lattice == 1 ? 2 : 1) > kAutoPairMaxN) return false;
  }
  return true;
}

extern "C" vmc_status vmc_default_params(vmc_solver_params* p) {
  if (!p) return VMC_ERR_INVALID;
  p->drop_tol = 1e-4;
  p->permtol = 0.5;
  p->lfil_extra = -1;
  p->gmres_m = 30;
  p->max_restarts = 10;
  p->inner_rtol = 0.0;
  p->ratio_tol = 1e-12;
  p->N_max = 100.0;
  p->slow_factor = 4.0;
  p->max_updates = -1;
  p->precision = VMC_PREC_MIXED;
  p->engine = VMC_ENGINE_PERSISTENT;
  p->block_threads = 0;
  p->sm_refresh = 1;
  p->refactor_lag = -1;
  p->refactor_reorder = 0;
  p->trisolve = 0;
  p->graphs = 1;
  p->trigger_rtol = 1e-6;
  p->trigger_its = 40;
  p->sweep_moves = 0;
  p->ilutp_variant = 0;
  p->trisolve_warp_rows = 0;
  p->trisolve_group = 8;
  p->trisolve_row_cap = 0;
  p->trisolve_lane_entries = 0;
  return VMC_OK;
}

namespace {
struct Carve {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t o = off;
    off += count * sizeof(T);
    return o;
  }
};
}  // namespace

// Dense engine (explicit inverse + Sherman-Morrison, Sec. 1): per walker the sparse
// rows (orbital columns, identity layout), the n x n inverse and two work vectors.
static vmc_status create_dense(vmc_ctx* ctx, const std::vector<Layout>& lay) {
  const int nw = ctx->nw;
  ctx->dense = true;
  ctx->threads = ctx->prm.block_threads ? ctx->prm.block_threads : 256;
  ctx->smem = 0;
  std::vector<std::vector<size_t>> offs(nw);
  Carve cv;
  ctx->hw.resize(nw);
  long long base = 0;
  for (int w = 0; w < nw; ++w) {
    const Layout& L = lay[w];
    const int n = L.n, cap = L.cap;
    auto& o = offs[w];
    o.push_back(cv.take<double>((size_t)n * 3));   // Z
    o.push_back(cv.take<int>(n));                  // identity column map
    o.push_back(cv.take<double>((size_t)n * 3));   // R
    o.push_back(cv.take<int>((size_t)n * cap));    // a_col
    o.push_back(cv.take<double>((size_t)n * cap)); // a_val
    o.push_back(cv.take<int>(n));                  // a_len
    o.push_back(cv.take<double>((size_t)n * n));   // B
    o.push_back(cv.take<double>(n));               // dcol
    o.push_back(cv.take<double>(n));               // drow
    o.push_back(cv.take<int>(n));                  // dpiv
    Walker& W = ctx->hw[w];
    std::memset(&W, 0, sizeof(W));
    const vmc_system& s = ctx->sys[w];
    W.n = n; W.K = s.K; W.lattice = s.lattice; W.cap = cap; W.per = L.per;
    W.a = s.a; W.kappa = s.kappa; W.rc = s.r_c; W.rc2 = s.r_c * s.r_c; W.L = s.K * s.a;
    W.log_base = base;
    base += n;
    ctx->max_n = std::max(ctx->max_n, n);
  }
  ctx->total_n = base;
  const size_t ctl_off = cv.take<Ctl>(nw);
  const size_t walk_off = cv.take<Walker>(nw);
  ctx->arena_bytes = cv.off + 256;
  cudaError_t e = cudaMalloc((void**)&ctx->arena, ctx->arena_bytes);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc arena");
  e = cudaMemsetAsync(ctx->arena, 0, ctx->arena_bytes, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemset arena");
  char* A = ctx->arena;
  ctx->dCtl = (Ctl*)(A + ctl_off);
  ctx->dW = (Walker*)(A + walk_off);
  for (int w = 0; w < nw; ++w) {
    const auto& o = offs[w];
    Walker& W = ctx->hw[w];
    const int n = W.n;
    W.Z = (const double*)(A + o[0]);
    W.col_of_orb = (const int*)(A + o[1]);
    W.orb_of_col = (const int*)(A + o[1]);
    W.R = (double*)(A + o[2]);
    W.a_col = (int*)(A + o[3]);
    W.a_val = (double*)(A + o[4]);
    W.a_len = (int*)(A + o[5]);
    W.Bd = (double*)(A + o[6]);
    W.dcol = (double*)(A + o[7]);
    W.drow = (double*)(A + o[8]);
    W.dpiv = (int*)(A + o[9]);
    W.ctl = ctx->dCtl + w;
    std::vector<int> ident(n);
    for (int j = 0; j < n; ++j) ident[j] = j;
    e = cudaMemcpyAsync((void*)W.Z, lay[w].Z.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)W.col_of_orb, ident.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upload layout");
  }
  e = cudaMemcpyAsync(ctx->dW, ctx->hw.data(), sizeof(Walker) * nw, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_seeds, sizeof(uint64_t) * nw);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload walkers");
  ctx->pending.assign(nw, 0);
  return VMC_OK;
}

extern "C" vmc_status vmc_create(const vmc_system* systems, int n_walkers, const vmc_solver_params* params,
                                 void* stream, vmc_ctx** out) {
  if (!out) return VMC_ERR_INVALID;
  *out = nullptr;
  if (!systems || n_walkers <= 0 || n_walkers > 65535) return VMC_ERR_INVALID;
  vmc_ctx* ctx = new vmc_ctx();
  ctx->nw = n_walkers;
  ctx->sys.assign(systems, systems + n_walkers);
  if (params) ctx->prm = *params; else vmc_default_params(&ctx->prm);
  vmc_solver_params& p = ctx->prm;
  ctx->stream = (cudaStream_t)stream;
  auto bad = [&](const std::string& m) { ctx->err = m; return VMC_ERR_INVALID; };
  vmc_status st = VMC_OK;
  if (p.gmres_m < 1 || p.gmres_m > kMaxM) st = bad("gmres_m must be in [1, 40]");
  else if (p.max_updates < -1 || p.max_updates > kMaxUpd) st = bad("max_updates must be -1 or in [0, 128]");
  else if (p.precision != VMC_PREC_FP64 && p.precision != VMC_PREC_MIXED && p.precision != VMC_PREC_MIXED_F32ILU)
    st = bad("precision");
  else if (p.engine < VMC_ENGINE_PLAIN || p.engine > VMC_ENGINE_DENSE_SM) st = bad("engine");
  else if (p.engine == VMC_ENGINE_DENSE_SM && p.precision != VMC_PREC_FP64) st = bad("the dense engine is FP64 only");
  else if (p.sm_refresh < 0) st = bad("sm_refresh must be >= 0");
  else if (p.block_threads != 0 && (p.block_threads < 64 || p.block_threads > kMaxThreads || p.block_threads % 32))
    st = bad("block_threads must be 0 or a multiple of 32 in [64, 256]");
  else if (!(p.drop_tol >= 0.0) || !(p.permtol >= 0.0) || p.max_restarts < 0) st = bad("ILUTP/GMRES parameters");
  else if (p.refactor_lag < -1) st = bad("refactor_lag must be >= -1");
  else if (p.trisolve < 0 || p.trisolve > 1) st = bad("trisolve must be 0 or 1");
  else if (p.sweep_moves < 0) st = bad("sweep_moves must be >= 0");
  else if (p.ilutp_variant < 0 || p.ilutp_variant > 2) st = bad("ilutp_variant must be 0, 1 or 2");
  else if (p.trisolve_warp_rows < 0 || p.trisolve_warp_rows > 32) st = bad("trisolve_warp_rows must be in [0, 32]");
  else if (p.trisolve_group < 0 || p.trisolve_group > 64) st = bad("trisolve_group must be in [0, 64]");
  else if (p.trisolve_row_cap < 0 || p.trisolve_row_cap > 480) st = bad("trisolve_row_cap must be in [0, 480]");
  else if (p.trisolve_lane_entries < 0 || p.trisolve_lane_entries > 64) st = bad("trisolve_lane_entries must be in [0, 64]");
  else if (!(p.trigger_rtol < 1.0)) st = bad("trigger_rtol must be below 1");
  if (st != VMC_OK) { *out = ctx; return st; }
  ctx->fp64 = p.precision == VMC_PREC_FP64;
  ctx->threads = p.block_threads ? p.block_threads : 256;
  ctx->P.drop_tol = p.drop_tol;
  ctx->P.permtol = p.permtol;
  ctx->P.lfil_extra = p.lfil_extra;
  ctx->P.m = p.gmres_m;
  ctx->P.max_restarts = p.max_restarts;
  ctx->P.inner_rtol = p.inner_rtol > 0.0 ? p.inner_rtol : (ctx->fp64 ? 1e-10 : 1e-5);
  ctx->P.ratio_tol = p.ratio_tol > 0.0 ? p.ratio_tol : 1e-12;
  ctx->P.ilu64 = p.precision != VMC_PREC_MIXED_F32ILU;
  ctx->P.N_max = p.N_max;
  ctx->P.slow_factor = p.slow_factor;
  ctx->P.trig_rtol = p.trigger_rtol > 0.0 ? p.trigger_rtol : 1e-6;
  ctx->P.trig_its = p.trigger_its > 0 ? p.trigger_its : 40;
  ctx->P.step_limit = p.sweep_moves;
  ctx->P.ilu_variant = p.ilutp_variant;
  ctx->P.warp_rows = p.trisolve_warp_rows;
  ctx->row_cap = p.trisolve_row_cap;
  ctx->P.lane_entries = p.trisolve_lane_entries > 0 ? p.trisolve_lane_entries : (ctx->fp64 ? 8 : 2);
  ctx->P.tri_group = p.trisolve == 1 ? 1 : std::max(1, p.trisolve_group);  // the sync-free solves read levels
  {
    // background refactorisation (persistent engine) when asked for, or by default when
    // every walker pair fits and no system is larger than kAutoPairMaxN; the chain length
    // defaults to 64 with it (adopted every 32 accepts) and to 128 without (in-line
    // refactorisations are the costlier)
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const bool fits = auto_pairs_fit(systems, n_walkers, nsm);
    const bool bg = p.engine == VMC_ENGINE_PERSISTENT && (p.refactor_lag > 0 || (p.refactor_lag < 0 && fits));
    p.max_updates = p.max_updates >= 0 ? p.max_updates : (bg ? 64 : 128);
    int lag = 0;
    if (bg) lag = std::min(p.refactor_lag > 0 ? p.refactor_lag : p.max_updates / 2, p.max_updates / 2);
    ctx->P.max_updates = p.max_updates;
    ctx->P.af_lag = std::max(lag, 0);
    ctx->P.af_reorder = p.refactor_reorder ? 1 : 0;
    ctx->pair = ctx->P.af_lag > 0;
  }

  // layouts (one per distinct system)
  std::vector<Layout> lay(n_walkers);
  for (int w = 0; w < n_walkers; ++w) {
    const vmc_system& s = systems[w];
    bool reused = false;
    for (int v = 0; v < w && !reused; ++v)
      if (!std::memcmp(&systems[v], &s, sizeof(vmc_system))) { lay[w] = lay[v]; reused = true; }
    if (reused) continue;
    const char* why = "";
    if (make_layout(s.K, s.lattice, s.a, s.r_c, lay[w], &why) || !(s.kappa > 0.0)) {
      ctx->err = std::string("walker ") + std::to_string(w) + ": " + (s.kappa > 0.0 ? why : "kappa must be positive");
      *out = ctx;
      return VMC_ERR_INVALID;
    }
    if (p.engine != VMC_ENGINE_DENSE_SM && !rows_fit_slot(lay[w].cap, p.lfil_extra, p.trisolve_row_cap)) {
      ctx->err = std::string("walker ") + std::to_string(w) + ": factor rows longer than a stream slot (r_c or lfil_extra too large)";
      *out = ctx;
      return VMC_ERR_INVALID;
    }
  }
  if (p.engine == VMC_ENGINE_DENSE_SM) {
    vmc_status ds = create_dense(ctx, lay);
    *out = ctx;
    return ds;
  }
  // carve one arena
  const size_t Tsz = ctx->fp64 ? sizeof(double) : sizeof(float);
  const int m = p.gmres_m, mu = std::max(1, p.max_updates);
  std::vector<std::vector<size_t>> offs(n_walkers);
  Carve cv;
  ctx->hw.resize(n_walkers);
  long long base = 0;
  for (int w = 0; w < n_walkers; ++w) {
    const Layout& L = lay[w];
    const int n = L.n, cap = L.cap;
    const int pmax = p.lfil_extra >= 0 ? p.lfil_extra : (cap + 1) / 2;
    const int capLU = (cap + pmax + 2 + 3) / 4 * 4;  // rows of 16-byte multiples (bulk copies)
    const int exmax = expanded_row_cap(capLU, p.trisolve_row_cap);
    auto& o = offs[w];
    o.push_back(cv.take<double>((size_t)n * 3));       // 0 Z
    o.push_back(cv.take<int>(n));                      // 1 col_of_orb
    o.push_back(cv.take<int>(n));                      // 2 orb_of_col
    o.push_back(cv.take<double>((size_t)n * 3));       // 3 R
    o.push_back(cv.take<int>(n));                      // 4 row_of_part
    o.push_back(cv.take<int>(n));                      // 5 part_of_row
    o.push_back(cv.take<int>((size_t)n * cap));        // 6 a_col
    o.push_back(cv.take<double>((size_t)n * cap));     // 7 a_val
    o.push_back(cv.take<float>((size_t)n * cap));      // 8 a_val32
    o.push_back(cv.take<int>(n));                      // 9 a_len
    o.push_back(cv.take<int>((size_t)n * capLU));      // 10 l_col
    o.push_back(cv.take<double>((size_t)n * capLU));   // 11 l_val64
    const size_t sbytes = (size_t)n * (256 + 12 * (size_t)std::max(capLU, exmax));
    o.push_back(cv.take<unsigned char>(sbytes));       // 12 lstream
    o.push_back(cv.take<int>(n));                      // 13 l_len
    o.push_back(cv.take<int>((size_t)n * capLU));      // 14 u_col
    o.push_back(cv.take<double>((size_t)n * capLU));   // 15 u_val64
    o.push_back(cv.take<unsigned char>(sbytes));       // 16 ustream
    o.push_back(cv.take<int>(n));                      // 17 u_len
    o.push_back(cv.take<double>(n));                   // 18 u_dinv64
    o.push_back(cv.take<int2>(2 * (size_t)n + 2));     // 19 lchunk | uchunk
    o.push_back(cv.take<int>(n));                      // 20 perm
    o.push_back(cv.take<int>(n));                      // 21 iperm
    o.push_back(cv.take<int>(n));                      // 22 lev_l
    o.push_back(cv.take<int>(n));                      // 23 lev_u
    o.push_back(cv.take<int>(n + 1));                  // 24 l_lvl_ptr
    o.push_back(cv.take<int>(n));                      // 25 l_lvl_rows
    o.push_back(cv.take<int>(n + 1));                  // 26 u_lvl_ptr
    o.push_back(cv.take<int>(n));                      // 27 u_lvl_rows
    o.push_back(cv.take<int>(n + 1));                  // 28 lvl_cur
    o.push_back(cv.take<double>(n));                   // 29 wrow
    o.push_back(cv.take<int>(n));                      // 30 wpos
    o.push_back(cv.take<int>(n));                      // 31 gP
    o.push_back(cv.take<int>(n));                      // 32 gQ
    o.push_back(cv.take<char>((size_t)((mu + 3) / 4 * 4) * n * Tsz)); // 33 upd_z (transposed)
    o.push_back(cv.take<int>((size_t)mu * kMaxU));     // 34 upd_ucol
    o.push_back(cv.take<char>((size_t)mu * kMaxU * Tsz));  // 35 upd_uval
    o.push_back(cv.take<int>(mu));                     // 36 upd_ulen
    o.push_back(cv.take<double>((size_t)kMaxUpd * kMaxUpd));  // 37 upd_G
    o.push_back(cv.take<char>((size_t)(m + 1) * n * Tsz));    // 38 V
    o.push_back(cv.take<char>((size_t)m * n * Tsz));          // 39 Zk
    o.push_back(cv.take<char>((size_t)3 * n * Tsz));          // 40 tv (three solve vectors)
    o.push_back(cv.take<double>(n));                   // 41 x64
    o.push_back(cv.take<double>(n));                   // 42 r64
    o.push_back(cv.take<int>(cap));                    // 43 pend_acol
    o.push_back(cv.take<double>(cap));                 // 44 pend_aval
    o.push_back(cv.take<int>(kMaxU));                  // 45 pend_ucol
    o.push_back(cv.take<double>(kMaxU));               // 46 pend_uval
    o.push_back(cv.take<int4>(n + 1));                 // 47 chunk_meta
    o.push_back(cv.take<int>(n + 1));                  // 48 lvl_nchunk
    o.push_back(cv.take<int4>(2 * (size_t)n + 2));     // 49 seg_meta
    if (ctx->pair) {
      // second factor set (same order as offsets 10-30, 47-49), then the snapshot of A
      o.push_back(cv.take<int>((size_t)n * capLU));    // 50 l_col
      o.push_back(cv.take<double>((size_t)n * capLU)); // 51 l_val64
      o.push_back(cv.take<unsigned char>(sbytes));     // 52 lstream
      o.push_back(cv.take<int>(n));                    // 53 l_len
      o.push_back(cv.take<int>((size_t)n * capLU));    // 54 u_col
      o.push_back(cv.take<double>((size_t)n * capLU)); // 55 u_val64
      o.push_back(cv.take<unsigned char>(sbytes));     // 56 ustream
      o.push_back(cv.take<int>(n));                    // 57 u_len
      o.push_back(cv.take<double>(n));                 // 58 u_dinv64
      o.push_back(cv.take<int2>(2 * (size_t)n + 2));   // 59 lchunk | uchunk
      o.push_back(cv.take<int>(n));                    // 60 perm
      o.push_back(cv.take<int>(n));                    // 61 iperm
      o.push_back(cv.take<int>(n));                    // 62 lev_l
      o.push_back(cv.take<int>(n));                    // 63 lev_u
      o.push_back(cv.take<int>(n + 1));                // 64 l_lvl_ptr
      o.push_back(cv.take<int>(n));                    // 65 l_lvl_rows
      o.push_back(cv.take<int>(n + 1));                // 66 u_lvl_ptr
      o.push_back(cv.take<int>(n));                    // 67 u_lvl_rows
      o.push_back(cv.take<int>(n + 1));                // 68 lvl_cur
      o.push_back(cv.take<double>(n));                 // 69 wrow
      o.push_back(cv.take<int>(n));                    // 70 wpos
      o.push_back(cv.take<int4>(n + 1));               // 71 chunk_meta
      o.push_back(cv.take<int>(n + 1));                // 72 lvl_nchunk
      o.push_back(cv.take<int4>(2 * (size_t)n + 2));   // 73 seg_meta
      o.push_back(cv.take<int>(n));                    // 74 snap_len
      o.push_back(cv.take<int>((size_t)n * cap));      // 75 snap_col
      o.push_back(cv.take<double>((size_t)n * cap));   // 76 snap_val
      o.push_back(cv.take<int>(n));                    // 77 snap_part
      o.push_back(cv.take<double>((size_t)n * 3));     // 78 snap_R
      o.push_back(cv.take<int>(n));                    // 79 snap_rop
      o.push_back(cv.take<int>(n));                    // 80 gP of the factor CTA
      o.push_back(cv.take<int>(n));                    // 81 gQ of the factor CTA
    }
    o.push_back(cv.take<double2>(n));                  // u_head of factor set 0 (then of set 1)
    if (ctx->pair) o.push_back(cv.take<double2>(n));
    for (int sset = 0; sset < (ctx->pair ? 2 : 1); ++sset) {  // expanded rows of each factor set
      o.push_back(cv.take<int>(n));                      // ex_len
      o.push_back(cv.take<int>((size_t)n * exmax));      // ex_col
      o.push_back(cv.take<double>((size_t)n * exmax));   // ex_val
      o.push_back(cv.take<int>(n + 1));                  // gptr
    }
    Walker& W = ctx->hw[w];
    std::memset(&W, 0, sizeof(W));
    W.n = n; W.K = systems[w].K; W.lattice = systems[w].lattice; W.cap = cap; W.capLU = capLU;
    W.m = m; W.mu = mu; W.mu4 = (mu + 3) / 4 * 4; W.per = L.per;
    W.a = systems[w].a; W.kappa = systems[w].kappa; W.rc = systems[w].r_c;
    W.rc2 = systems[w].r_c * systems[w].r_c; W.L = systems[w].K * systems[w].a;
    W.log_base = base;
    base += n;
    ctx->max_n = std::max(ctx->max_n, n);
  }
  ctx->total_n = base;
  {
    // shared-memory plan: the triangular-solve vector in shared memory when it fits,
    // and a ring of 2..8 chunk slots; aim for 2 CTAs per SM when walkers outnumber SMs
    int dev = 0, optin = 0, per_sm = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int stat = kernel_static_smem(ctx->fp64);
    if (optin <= 0 || per_sm <= 0 || nsm <= 0 || stat <= 0) {
      *out = ctx;
      return fail(ctx, VMC_ERR_CUDA, "no usable CUDA device (shared-memory attributes unavailable)");
    }
    // grouped solves keep two vectors in shared memory; when two do not fit, one (the
    // level-by-level solve in place) -- walkers whose two vectors fit it still group
    const int ybytes1 = (int)(((size_t)ctx->max_n * Tsz + 127) / 128 * 128);
    const int ybytes = ctx->P.tri_group > 1 ? (int)(((size_t)2 * ctx->max_n * Tsz + 127) / 128 * 128) : ybytes1;
    const int budget1 = optin - stat;
    const int budget2 = per_sm / 2 - 1024 - stat;
    int budget = budget1;
    if (n_walkers > nsm && budget2 >= ybytes + 2 * kSlotBytes) budget = budget2;
    plan_smem(ybytes, budget, ctx->P, p.trisolve == 1);
    if (!ctx->P.y_smem && ybytes != ybytes1) plan_smem(ybytes1, budget, ctx->P, p.trisolve == 1);
    ctx->smem = (size_t)ctx->P.dsm_bytes;
  }
  const size_t ctl_off = cv.take<Ctl>(n_walkers);
  const size_t walk_off = cv.take<Walker>(n_walkers);
  const size_t energy_off = cv.take<double>(n_walkers);
  const size_t budget_off = cv.take<unsigned long long>(1);
  const size_t shadow_off = ctx->pair ? cv.take<Ctl>(n_walkers) : 0;
  const size_t walk1_off = ctx->pair ? cv.take<Walker>(n_walkers) : 0;
  const size_t walkf_off = ctx->pair ? cv.take<Walker>(2 * (size_t)n_walkers) : 0;
  ctx->arena_bytes = cv.off + 256;
  cudaError_t e = cudaMalloc((void**)&ctx->arena, ctx->arena_bytes);
  if (e != cudaSuccess) { *out = ctx; return cuda_fail(ctx, e, "cudaMalloc arena"); }
  e = cudaMemsetAsync(ctx->arena, 0, ctx->arena_bytes, ctx->stream);
  if (e != cudaSuccess) { *out = ctx; return cuda_fail(ctx, e, "cudaMemset arena"); }
  char* A = ctx->arena;
  ctx->dCtl = (Ctl*)(A + ctl_off);
  ctx->dW = (Walker*)(A + walk_off);
  ctx->d_energy = (double*)(A + energy_off);
  ctx->d_budget = (unsigned long long*)(A + budget_off);
  for (int w = 0; w < n_walkers; ++w) {
    const auto& o = offs[w];
    Walker& W = ctx->hw[w];
    W.Z = (const double*)(A + o[0]);
    W.col_of_orb = (const int*)(A + o[1]);
    W.orb_of_col = (const int*)(A + o[2]);
    W.R = (double*)(A + o[3]);
    W.row_of_part = (int*)(A + o[4]);
    W.part_of_row = (int*)(A + o[5]);
    W.a_col = (int*)(A + o[6]);
    W.a_val = (double*)(A + o[7]);
    W.a_val32 = (float*)(A + o[8]);
    W.a_len = (int*)(A + o[9]);
    W.l_col = (int*)(A + o[10]);
    W.l_val64 = (double*)(A + o[11]);
    W.lstream = (unsigned char*)(A + o[12]);
    W.l_len = (int*)(A + o[13]);
    W.u_col = (int*)(A + o[14]);
    W.u_val64 = (double*)(A + o[15]);
    W.ustream = (unsigned char*)(A + o[16]);
    W.u_len = (int*)(A + o[17]);
    W.u_dinv64 = (double*)(A + o[18]);
    W.lchunk = (int2*)(A + o[19]);
    W.uchunk = W.lchunk + (W.n + 1);
    W.perm = (int*)(A + o[20]);
    W.iperm = (int*)(A + o[21]);
    W.lev_l = (int*)(A + o[22]);
    W.lev_u = (int*)(A + o[23]);
    W.l_lvl_ptr = (int*)(A + o[24]);
    W.l_lvl_rows = (int*)(A + o[25]);
    W.u_lvl_ptr = (int*)(A + o[26]);
    W.u_lvl_rows = (int*)(A + o[27]);
    W.lvl_cur = (int*)(A + o[28]);
    W.wrow = (double*)(A + o[29]);
    W.wpos = (int*)(A + o[30]);
    W.gP = (int*)(A + o[31]);
    W.gQ = (int*)(A + o[32]);
    W.upd_z = (void*)(A + o[33]);
    W.upd_ucol = (int*)(A + o[34]);
    W.upd_uval = (void*)(A + o[35]);
    W.upd_ulen = (int*)(A + o[36]);
    W.upd_G = (double*)(A + o[37]);
    W.V = (void*)(A + o[38]);
    W.Zk = (void*)(A + o[39]);
    W.tv = (void*)(A + o[40]);
    W.x64 = (double*)(A + o[41]);
    W.r64 = (double*)(A + o[42]);
    W.pend_acol = (int*)(A + o[43]);
    W.pend_aval = (double*)(A + o[44]);
    W.pend_ucol = (int*)(A + o[45]);
    W.pend_uval = (double*)(A + o[46]);
    W.chunk_meta = (int4*)(A + o[47]);
    W.lvl_nchunk = (int*)(A + o[48]);
    W.seg_meta = (int4*)(A + o[49]);
    W.u_head = (double2*)(A + o[ctx->pair ? 82 : 50]);
    {
      const size_t e0 = ctx->pair ? 84 : 51;
      W.exmax = expanded_row_cap(W.capLU, ctx->row_cap);
      W.ex_len = (int*)(A + o[e0]);
      W.ex_col = (int*)(A + o[e0 + 1]);
      W.ex_val = (double*)(A + o[e0 + 2]);
      W.gptr = (int*)(A + o[e0 + 3]);
    }
    W.ctl = ctx->dCtl + w;
    const Layout& L = lay[w];
    e = cudaMemcpyAsync((void*)W.Z, L.Z.data(), sizeof(double) * L.Z.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)W.col_of_orb, L.col_of_orb.data(), sizeof(int) * L.n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)W.orb_of_col, L.orb_of_col.data(), sizeof(int) * L.n, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) { *out = ctx; return cuda_fail(ctx, e, "upload layout"); }
  }
  if (ctx->pair) {
    // views: hw1 = the walker with factor set 1; hwf[2w + s] = the factor CTA's view
    // (factor set s, matrix = the snapshot, controller = the shadow)
    ctx->dShadow = (Ctl*)(A + shadow_off);
    ctx->dW1 = (Walker*)(A + walk1_off);
    ctx->dWf = (Walker*)(A + walkf_off);
    ctx->hw1 = ctx->hw;
    ctx->hwf.assign(2 * (size_t)n_walkers, Walker{});
    for (int w = 0; w < n_walkers; ++w) {
      const auto& o = offs[w];
      Walker& W0 = ctx->hw[w];
      Walker& W1 = ctx->hw1[w];
      W1.l_col = (int*)(A + o[50]);
      W1.l_val64 = (double*)(A + o[51]);
      W1.lstream = (unsigned char*)(A + o[52]);
      W1.l_len = (int*)(A + o[53]);
      W1.u_col = (int*)(A + o[54]);
      W1.u_val64 = (double*)(A + o[55]);
      W1.ustream = (unsigned char*)(A + o[56]);
      W1.u_len = (int*)(A + o[57]);
      W1.u_dinv64 = (double*)(A + o[58]);
      W1.lchunk = (int2*)(A + o[59]);
      W1.uchunk = W1.lchunk + (W1.n + 1);
      W1.perm = (int*)(A + o[60]);
      W1.iperm = (int*)(A + o[61]);
      W1.lev_l = (int*)(A + o[62]);
      W1.lev_u = (int*)(A + o[63]);
      W1.l_lvl_ptr = (int*)(A + o[64]);
      W1.l_lvl_rows = (int*)(A + o[65]);
      W1.u_lvl_ptr = (int*)(A + o[66]);
      W1.u_lvl_rows = (int*)(A + o[67]);
      W1.lvl_cur = (int*)(A + o[68]);
      W1.wrow = (double*)(A + o[69]);
      W1.wpos = (int*)(A + o[70]);
      W1.chunk_meta = (int4*)(A + o[71]);
      W1.lvl_nchunk = (int*)(A + o[72]);
      W1.seg_meta = (int4*)(A + o[73]);
      W1.u_head = (double2*)(A + o[83]);
      W1.ex_len = (int*)(A + o[88]);
      W1.ex_col = (int*)(A + o[89]);
      W1.ex_val = (double*)(A + o[90]);
      W1.gptr = (int*)(A + o[91]);
      W0.snap_len = (int*)(A + o[74]);
      W0.snap_col = (int*)(A + o[75]);
      W0.snap_val = (double*)(A + o[76]);
      W0.snap_part = (int*)(A + o[77]);
      W0.snap_R = (double*)(A + o[78]);
      W0.snap_rop = (int*)(A + o[79]);
      W0.shadow = ctx->dShadow + w;
      W0.set_id = 0;
      W1.set_id = 1;
      for (int sset = 0; sset < 2; ++sset) {
        Walker F = sset ? W1 : W0;
        F.a_col = W0.snap_col;
        F.a_val = W0.snap_val;
        F.a_len = W0.snap_len;
        F.part_of_row = W0.snap_part;
        F.row_of_part = W0.snap_rop;
        F.R = W0.snap_R;
        F.gP = (int*)(A + o[80]);
        F.gQ = (int*)(A + o[81]);
        F.ctl = W0.shadow;
        F.alt = nullptr;
        F.fact[0] = F.fact[1] = nullptr;
        ctx->hwf[2 * (size_t)w + sset] = F;
      }
      W0.alt = ctx->dW1 + w;
      W0.fact[0] = ctx->dWf + 2 * (size_t)w;
      W0.fact[1] = ctx->dWf + 2 * (size_t)w + 1;
      W1.alt = nullptr;
      W1.fact[0] = W0.fact[0];
      W1.fact[1] = W0.fact[1];
      W1.snap_len = W0.snap_len; W1.snap_col = W0.snap_col; W1.snap_val = W0.snap_val; W1.snap_part = W0.snap_part;
      W1.snap_R = W0.snap_R; W1.snap_rop = W0.snap_rop;
      W1.shadow = W0.shadow;
    }
    e = cudaMemcpyAsync(ctx->dW1, ctx->hw1.data(), sizeof(Walker) * n_walkers, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ctx->dWf, ctx->hwf.data(), sizeof(Walker) * 2 * n_walkers, cudaMemcpyHostToDevice,
                          ctx->stream);
    if (e != cudaSuccess) { *out = ctx; return cuda_fail(ctx, e, "upload walker views"); }
  }
  e = cudaMemcpyAsync(ctx->dW, ctx->hw.data(), sizeof(Walker) * n_walkers, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_seeds, sizeof(uint64_t) * n_walkers);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) { *out = ctx; return cuda_fail(ctx, e, "upload walkers"); }
  ctx->pending.assign(n_walkers, 0);
  *out = ctx;
  return VMC_OK;
}

extern "C" vmc_status vmc_destroy(vmc_ctx* ctx) {
  if (!ctx) return VMC_ERR_INVALID;
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->d_sweep) cudaFree(ctx->d_sweep);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->d_seeds) cudaFree(ctx->d_seeds);
  if (ctx->d_acc) cudaFree(ctx->d_acc);
  if (ctx->d_ratio) cudaFree(ctx->d_ratio);
  delete ctx;
  return VMC_OK;
}

extern "C" const char* vmc_last_error(const vmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
extern "C" int vmc_walker_n(const vmc_ctx* ctx, int walker) {
  if (!ctx || walker < 0 || walker >= ctx->nw) return -1;
  return ctx->hw[walker].n;
}
extern "C" int64_t vmc_sweep_count(const vmc_ctx* ctx) { return ctx ? ctx->sweeps : -1; }
extern "C" vmc_status vmc_set_sweep_count(vmc_ctx* ctx, int64_t sweeps) {
  if (!ctx || sweeps < 0) return VMC_ERR_INVALID;
  ctx->sweeps = sweeps;
  return VMC_OK;
}

static vmc_status check_walker_status(vmc_ctx* ctx) {
  std::vector<Ctl> h(ctx->nw);
  CK(cudaMemcpyAsync(h.data(), ctx->dCtl, sizeof(Ctl) * ctx->nw, cudaMemcpyDeviceToHost, ctx->stream), "read status");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  for (int w = 0; w < ctx->nw; ++w)
    if (h[w].status != ST_OK)
      return fail(ctx, (vmc_status)h[w].status, "walker " + std::to_string(w) + " failed with status " + std::to_string(h[w].status));
  return VMC_OK;
}

static vmc_status setup_all(vmc_ctx* ctx, int w0, int nwalk) {
  if (ctx->dense) CK(launch_dense_setup(cfg(ctx), ctx->dW + w0, nwalk), "dense setup kernel");
  else CK(launch_setup(cfg(ctx), ctx->dW, w0, nwalk, ctx->P), "setup kernel");
  for (int w = w0; w < w0 + nwalk; ++w) ctx->pending[w] = 0;
  ctx->ready = true;
  return check_walker_status(ctx);
}

extern "C" vmc_status vmc_init_positions(vmc_ctx* ctx, const uint64_t* seeds, double jitter) {
  if (!ctx || !seeds || !(jitter >= 0.0)) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  CK(cudaMemcpyAsync(ctx->d_seeds, seeds, sizeof(uint64_t) * ctx->nw, cudaMemcpyHostToDevice, ctx->stream), "seeds");
  CK(cudaMemsetAsync(ctx->dCtl, 0, sizeof(Ctl) * ctx->nw, ctx->stream), "reset walkers");
  CK(launch_init_positions(cfg(ctx), ctx->dW, ctx->nw, ctx->d_seeds, jitter), "init positions");
  return setup_all(ctx, 0, ctx->nw);
}

extern "C" vmc_status vmc_set_positions(vmc_ctx* ctx, int walker, const double* xyz) {
  if (!ctx || !xyz || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  const Walker& W = ctx->hw[walker];
  std::vector<double> r(xyz, xyz + (size_t)W.n * 3);
  for (double& v : r) {
    if (!std::isfinite(v)) return fail(ctx, VMC_ERR_INVALID, "non-finite position");
    double y = v - W.L * std::floor(v / W.L);
    if (y >= W.L) y -= W.L;
    v = y;
  }
  CK(cudaMemcpyAsync(W.R, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, ctx->stream), "positions");
  CK(cudaMemsetAsync(ctx->dCtl + walker, 0, sizeof(Ctl), ctx->stream), "reset walker");
  return setup_all(ctx, walker, 1);
}

extern "C" vmc_status vmc_set_positions_all(vmc_ctx* ctx, const double* xyz) {
  if (!ctx || !xyz) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  std::vector<double> r;
  size_t off = 0;
  for (int w = 0; w < ctx->nw; ++w) {
    const Walker& W = ctx->hw[w];
    r.assign(xyz + off, xyz + off + (size_t)W.n * 3);
    off += (size_t)W.n * 3;
    for (double& v : r) {
      if (!std::isfinite(v)) return fail(ctx, VMC_ERR_INVALID, "non-finite position (walker " + std::to_string(w) + ")");
      double y = v - W.L * std::floor(v / W.L);
      if (y >= W.L) y -= W.L;
      v = y;
    }
    CK(cudaMemcpyAsync(W.R, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, ctx->stream), "positions");
    // the pageable source is reused for the next walker: let the copy take it first
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  }
  CK(cudaMemsetAsync(ctx->dCtl, 0, sizeof(Ctl) * ctx->nw, ctx->stream), "reset walkers");
  return setup_all(ctx, 0, ctx->nw);
}

extern "C" vmc_status vmc_get_positions(vmc_ctx* ctx, int walker, double* xyz) {
  if (!ctx || !xyz || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  const Walker& W = ctx->hw[walker];
  CK(cudaMemcpyAsync(xyz, W.R, sizeof(double) * 3 * W.n, cudaMemcpyDeviceToHost, ctx->stream), "positions");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return VMC_OK;
}

static vmc_status ratio_impl(vmc_ctx* ctx, int walker, int k, const double r_new[3], double* ratio, double* grad,
                             double* lap) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || !r_new || !ratio || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  const Walker& W = ctx->hw[walker];
  if (k < 0 || k >= W.n) return fail(ctx, VMC_ERR_INVALID, "particle index out of range");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(r_new[d])) return fail(ctx, VMC_ERR_INVALID, "non-finite position");
  const bool want = grad || lap;
  CK(launch_ratio(cfg(ctx), ctx->dW, walker, ctx->P, k, r_new, want ? 1 : 0), "ratio kernel");
  Ctl h;
  CK(cudaMemcpyAsync(&h, ctx->dCtl + walker, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream), "read ratio");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  if (h.status != ST_OK) return fail(ctx, (vmc_status)h.status, "walker failed with status " + std::to_string(h.status));
  if (!h.pend_valid) { ctx->pending[walker] = 0; return fail(ctx, VMC_ERR_NOCONV, "solve did not converge"); }
  *ratio = h.pend_ratio;
  if (grad)
    for (int d = 0; d < 3; ++d) grad[d] = h.pend_grad[d];
  if (lap) *lap = h.pend_lap;
  ctx->pending[walker] = 1;
  return VMC_OK;
}

extern "C" vmc_status vmc_ratio(vmc_ctx* ctx, int walker, int k, const double r_new[3], double* ratio) {
  return ratio_impl(ctx, walker, k, r_new, ratio, nullptr, nullptr);
}

extern "C" vmc_status vmc_ratio_grad(vmc_ctx* ctx, int walker, int k, const double r_new[3], double* ratio,
                                     double grad[3], double* lap) {
  return ratio_impl(ctx, walker, k, r_new, ratio, grad, lap);
}

extern "C" vmc_status vmc_kinetic_energy(vmc_ctx* ctx, double* energy) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || !energy) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  CK(launch_kinetic(cfg(ctx), ctx->dW, ctx->nw, ctx->P, ctx->d_energy), "kinetic-energy kernel");
  CK(cudaMemcpyAsync(energy, ctx->d_energy, sizeof(double) * ctx->nw, cudaMemcpyDeviceToHost, ctx->stream), "energy");
  for (int w = 0; w < ctx->nw; ++w) ctx->pending[w] = 0;
  return check_walker_status(ctx);
}

extern "C" vmc_status vmc_accept(vmc_ctx* ctx, int walker) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->pending[walker]) return fail(ctx, VMC_ERR_STATE, "vmc_accept without a pending vmc_ratio");
  CK(launch_accept(cfg(ctx), ctx->dW, walker, ctx->P), "accept kernel");
  ctx->pending[walker] = 0;
  return check_walker_status(ctx);
}

static vmc_status ensure_logs(vmc_ctx* ctx, size_t entries) {
  if (entries <= ctx->log_cap) return VMC_OK;
  if (ctx->d_acc) cudaFree(ctx->d_acc);
  if (ctx->d_ratio) cudaFree(ctx->d_ratio);
  ctx->d_acc = nullptr;
  ctx->d_ratio = nullptr;
  ctx->log_cap = 0;
  CK(cudaMalloc((void**)&ctx->d_acc, entries), "log alloc");
  CK(cudaMalloc((void**)&ctx->d_ratio, entries * sizeof(double)), "log alloc");
  ctx->log_cap = entries;
  return VMC_OK;
}

// The launches of one sweep of the STEP or PLAIN engine (sweep index read from
// ctx->d_sweep when sweep_dev is set).
static cudaError_t step_launches(vmc_ctx* ctx, int n_sweeps, int s_local, long long s0, double sigma,
                                 const uint64_t* d_seeds, uint8_t* acc, double* ratio, const long long* sweep_dev,
                                 cudaStream_t stream) {
  LaunchCfg L = cfg(ctx);
  L.stream = stream;
  const int lim = ctx->P.step_limit;
  if (ctx->prm.engine == VMC_ENGINE_STEP) {
    const int qn = lim > 0 ? std::min(ctx->max_n, lim) : ctx->max_n;
    for (int q = 0; q < qn; ++q) {
      const cudaError_t e = launch_step(L, ctx->dW, 0, ctx->nw, ctx->P, q, n_sweeps, s_local, s0, sigma, d_seeds, acc,
                                        ratio, sweep_dev);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int w = 0; w < ctx->nw; ++w) {  // PLAIN: one walker per launch
    const int qn = lim > 0 ? std::min(ctx->hw[w].n, lim) : ctx->hw[w].n;
    for (int q = 0; q < qn; ++q) {
      const cudaError_t e = launch_step(L, ctx->dW, w, 1, ctx->P, q, n_sweeps, s_local, s0, sigma, d_seeds, acc, ratio,
                                        sweep_dev);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Capture (or reuse) the graph of one sweep: the step launches, then the advance of the
// device-side sweep index.  Captured on a private stream (the legacy default stream
// cannot be captured) and replayed on the context's stream.
static vmc_status sweep_graph(vmc_ctx* ctx, double sigma, const uint64_t* d_seeds, uint8_t* acc, double* ratio) {
  if (ctx->graph && ctx->g_seeds == d_seeds && ctx->g_acc == acc && ctx->g_ratio == ratio && ctx->g_sigma == sigma &&
      ctx->g_limit == ctx->P.step_limit)
    return VMC_OK;
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (!ctx->d_sweep) CK(cudaMalloc((void**)&ctx->d_sweep, sizeof(long long)), "sweep index");
  if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking), "capture stream");
  CK(prepare_step_kernels(cfg(ctx)), "step kernel attributes");
  CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal), "begin graph capture");
  cudaError_t e = step_launches(ctx, 1, 0, 0, sigma, d_seeds, acc, ratio, ctx->d_sweep, ctx->capture_stream);
  if (e == cudaSuccess) e = launch_next_sweep(ctx->d_sweep, ctx->capture_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(ctx->capture_stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ctx->graph = nullptr;
    return cuda_fail(ctx, e, "sweep graph");
  }
  ctx->g_seeds = d_seeds;
  ctx->g_acc = acc;
  ctx->g_ratio = ratio;
  ctx->g_sigma = sigma;
  ctx->g_limit = ctx->P.step_limit;
  return VMC_OK;
}

static vmc_status enqueue_sweeps(vmc_ctx* ctx, int n_sweeps, double sigma, const uint64_t* d_seeds, uint8_t* acc,
                                 double* ratio) {
  const LaunchCfg L = cfg(ctx);
  const long long s0 = ctx->sweeps;
  const int eng = ctx->prm.engine;
  if (eng == VMC_ENGINE_DENSE_SM) {
    CK(launch_dense_sweep(L, ctx->dW, ctx->nw, n_sweeps, s0, sigma, d_seeds, acc, ratio, ctx->prm.sm_refresh),
       "dense sweep kernel");
  } else if (eng == VMC_ENGINE_PERSISTENT && ctx->pair) {
    if (++ctx->launch_seq <= 0) ctx->launch_seq = 1;
    CK(launch_sweep_pair(L, ctx->dW, 0, ctx->nw, ctx->P, n_sweeps, s0, sigma, d_seeds, acc, ratio, ctx->launch_seq),
       "sweep kernel (walker pairs)");
  } else if (eng == VMC_ENGINE_PERSISTENT) {
    CK(launch_sweep(L, ctx->dW, 0, ctx->nw, ctx->P, n_sweeps, s0, sigma, d_seeds, acc, ratio), "sweep kernel");
  } else if (ctx->prm.graphs && (n_sweeps == 1 || (!acc && !ratio))) {
    // STEP / PLAIN: replay a captured graph of one sweep's launches per sweep
    vmc_status st = sweep_graph(ctx, sigma, d_seeds, acc, ratio);
    if (st != VMC_OK) return st;
    CK(launch_set_sweep(ctx->d_sweep, s0, ctx->stream), "sweep index");
    for (int s = 0; s < n_sweeps; ++s) CK(cudaGraphLaunch(ctx->graph, ctx->stream), "sweep graph");
  } else {  // STEP / PLAIN, launch by launch
    for (int s = 0; s < n_sweeps; ++s)
      CK(step_launches(ctx, n_sweeps, s, s0, sigma, d_seeds, acc, ratio, nullptr, ctx->stream), "step kernel");
  }
  ctx->sweeps += n_sweeps;
  return VMC_OK;
}

extern "C" vmc_status vmc_sweep(vmc_ctx* ctx, int n_sweeps, double sigma, const uint64_t* seeds, uint8_t* accept_log,
                                double* ratio_log) {
  if (!ctx || !seeds || n_sweeps < 0 || !(sigma >= 0.0)) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  if (n_sweeps == 0) return VMC_OK;
  const size_t entries = (size_t)n_sweeps * ctx->total_n;
  vmc_status st = VMC_OK;
  if (accept_log || ratio_log) {
    st = ensure_logs(ctx, entries);
    if (st != VMC_OK) return st;
  }
  CK(cudaMemcpyAsync(ctx->d_seeds, seeds, sizeof(uint64_t) * ctx->nw, cudaMemcpyHostToDevice, ctx->stream), "seeds");
  st = enqueue_sweeps(ctx, n_sweeps, sigma, ctx->d_seeds, accept_log ? ctx->d_acc : nullptr,
                      ratio_log ? ctx->d_ratio : nullptr);
  if (st != VMC_OK) return st;
  for (int w = 0; w < ctx->nw; ++w) ctx->pending[w] = 0;
  if (accept_log) CK(cudaMemcpyAsync(accept_log, ctx->d_acc, entries, cudaMemcpyDeviceToHost, ctx->stream), "accept log");
  if (ratio_log)
    CK(cudaMemcpyAsync(ratio_log, ctx->d_ratio, entries * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "ratio log");
  return check_walker_status(ctx);
}

extern "C" vmc_status vmc_sweep_async(vmc_ctx* ctx, int n_sweeps, double sigma, const uint64_t* seeds_dev,
                                      uint8_t* accept_log_dev, double* ratio_log_dev) {
  if (!ctx || !seeds_dev || n_sweeps < 0 || !(sigma >= 0.0)) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  if (n_sweeps == 0) return VMC_OK;
  for (int w = 0; w < ctx->nw; ++w) ctx->pending[w] = 0;
  return enqueue_sweeps(ctx, n_sweeps, sigma, seeds_dev, accept_log_dev, ratio_log_dev);
}

extern "C" vmc_status vmc_advance_async(vmc_ctx* ctx, int64_t total_moves, double sigma, const uint64_t* seeds_dev) {
  if (!ctx || !seeds_dev || total_moves < 0 || !(sigma >= 0.0)) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (ctx->prm.engine != VMC_ENGINE_PERSISTENT || ctx->dense)
    return fail(ctx, VMC_ERR_INVALID, "the budgeted advance needs the persistent engine");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  for (int w = 0; w < ctx->nw; ++w) ctx->pending[w] = 0;
  if (total_moves == 0) return VMC_OK;
  CK(cudaMemsetAsync(ctx->d_budget, 0, sizeof(unsigned long long), ctx->stream), "budget counter");
  Params P = ctx->P;
  P.budget_ctr = ctx->d_budget;
  P.budget_total = total_moves;
  const LaunchCfg L = cfg(ctx);
  if (ctx->pair) {
    if (++ctx->launch_seq <= 0) ctx->launch_seq = 1;
    CK(launch_sweep_pair(L, ctx->dW, 0, ctx->nw, P, 0, ctx->sweeps, sigma, seeds_dev, nullptr, nullptr,
                         ctx->launch_seq), "advance kernel (walker pairs)");
  } else {
    CK(launch_sweep(L, ctx->dW, 0, ctx->nw, P, 0, ctx->sweeps, sigma, seeds_dev, nullptr, nullptr), "advance kernel");
  }
  return VMC_OK;
}

extern "C" vmc_status vmc_advance(vmc_ctx* ctx, int64_t total_moves, double sigma, const uint64_t* seeds,
                                  int64_t* accepts_out) {
  if (!ctx || !seeds) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  CK(cudaMemcpyAsync(ctx->d_seeds, seeds, sizeof(uint64_t) * ctx->nw, cudaMemcpyHostToDevice, ctx->stream), "seeds");
  vmc_status st = vmc_advance_async(ctx, total_moves, sigma, ctx->d_seeds);
  if (st != VMC_OK) return st;
  st = check_walker_status(ctx);
  if (st != VMC_OK || !accepts_out) return st;
  std::vector<Ctl> h(ctx->nw);
  CK(cudaMemcpyAsync(h.data(), ctx->dCtl, sizeof(Ctl) * ctx->nw, cudaMemcpyDeviceToHost, ctx->stream), "accepts");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  for (int w = 0; w < ctx->nw; ++w) accepts_out[w] = h[w].accepts;
  return VMC_OK;
}

extern "C" vmc_status vmc_get_progress(vmc_ctx* ctx, int walker, int64_t* sweep, int* particle) {
  if (!ctx || !sweep || !particle || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  Ctl h;
  CK(cudaMemcpyAsync(&h, ctx->dCtl + walker, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream), "progress");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  *sweep = h.pos_valid ? h.pos_sweep : ctx->sweeps;
  *particle = h.pos_valid ? h.pos_k : 0;
  return VMC_OK;
}

extern "C" vmc_status vmc_synchronize(vmc_ctx* ctx) {
  if (!ctx) return VMC_ERR_INVALID;
  return check_walker_status(ctx);
}

extern "C" vmc_status vmc_get_stats(vmc_ctx* ctx, int walker, vmc_stats* out) {
  if (!ctx || !out || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  Ctl h;
  CK(cudaMemcpyAsync(&h, ctx->dCtl + walker, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream), "stats");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  std::memset(out, 0, sizeof(*out));
  out->proposals = h.proposals;
  out->accepts = h.accepts;
  out->solves = h.solves;
  out->inner_iterations = h.inner_its;
  out->first_pass_iterations = h.first_its;
  out->outer_passes = h.outer_passes;
  out->reorders = h.reorders;
  out->reorder_monitor = h.reorder_monitor;
  out->reorder_noconv = h.reorder_noconv;
  out->reorder_slow = h.reorder_slow;
  out->reorder_breakdown = h.reorder_breakdown;
  out->refactors_updates = h.refactors_updates;
  out->factorizations = h.factorizations;
  out->pivots = h.last_pivots;
  out->N_max_seen = h.N_max_seen;
  out->N_sum = h.N_sum;
  out->nnz_A = h.nnz_A;
  out->nnz_LU = h.nnz_LU;
  out->levels_L = h.nlev_l;
  out->levels_U = h.nlev_u;
  out->n_updates = h.n_upd;
  out->status = h.status;
  for (int b = 0; b < kHistBins; ++b) out->its_hist[b] = h.hist[b];
  for (int b = 0; b < 16; ++b) out->phase_cycles[b] = h.cyc[b];
  out->alg_bytes = h.alg_bytes;
  out->ilu_rows = h.ilu_rows;
  out->ilu_elims = h.ilu_elims;
  out->ilu_cand = h.ilu_cand;
  out->chunks_L = h.nchunk_l;
  out->chunks_U = h.nchunk_u;
  out->refactors_async = h.refactors_async;
  out->async_wait_cycles = h.af_wait_cyc;
  out->async_factor_cycles = h.af_factor_cyc;
  out->factor_set = h.active;
  out->async_lag = ctx->P.af_lag;
  out->max_updates = ctx->P.max_updates;
  out->reorders_skipped = h.reorder_skipped;
  out->trigger_iterations = h.trig_its;
  out->groups_L = h.ngrp_l;
  out->groups_U = h.ngrp_u;
  out->stream_bytes = h.stream_bytes;
  return VMC_OK;
}

extern "C" vmc_status vmc_reset_stats(vmc_ctx* ctx) {
  if (!ctx) return VMC_ERR_INVALID;
  std::vector<Ctl> h(ctx->nw);
  CK(cudaMemcpyAsync(h.data(), ctx->dCtl, sizeof(Ctl) * ctx->nw, cudaMemcpyDeviceToHost, ctx->stream), "stats");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  for (Ctl& c : h) {
    c.proposals = c.accepts = c.solves = c.inner_its = c.first_its = c.outer_passes = 0;
    c.reorders = c.reorder_monitor = c.reorder_noconv = c.reorder_slow = c.reorder_breakdown = 0;
    c.refactors_updates = c.factorizations = 0;
    c.N_max_seen = c.N_sum = 0.0;
    for (long long& b : c.hist) b = 0;
    for (long long& b : c.cyc) b = 0;
    c.alg_bytes = 0.0;
    c.ilu_rows = c.ilu_elims = c.ilu_cand = 0;
    c.refactors_async = c.af_wait_cyc = c.af_factor_cyc = 0;
    c.reorder_skipped = 0;
    c.trig_its = 0;
  }
  CK(cudaMemcpyAsync(ctx->dCtl, h.data(), sizeof(Ctl) * ctx->nw, cudaMemcpyHostToDevice, ctx->stream), "stats");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  return VMC_OK;
}

// ---- inspection ------------------------------------------------------------------
template <typename T>
static cudaError_t d2h(T* dst, const T* src, size_t count, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, sizeof(T) * count, cudaMemcpyDeviceToHost, s);
}

extern "C" vmc_status vmc_get_matrix(vmc_ctx* ctx, int walker, double* A_dense, int* part_of_row, int* orb_of_col) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  const Walker& W = ctx->hw[walker];
  const int n = W.n, cap = W.cap;
  std::vector<int> col((size_t)n * cap), len(n), por(n), ooc(n);
  std::vector<double> val((size_t)n * cap);
  CK(d2h(col.data(), W.a_col, col.size(), ctx->stream), "matrix");
  CK(d2h(val.data(), W.a_val, val.size(), ctx->stream), "matrix");
  CK(d2h(len.data(), W.a_len, len.size(), ctx->stream), "matrix");
  CK(d2h(por.data(), W.part_of_row, por.size(), ctx->stream), "matrix");
  CK(d2h(ooc.data(), W.orb_of_col, ooc.size(), ctx->stream), "matrix");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  if (A_dense) {
    std::fill(A_dense, A_dense + (size_t)n * n, 0.0);
    for (int r = 0; r < n; ++r) {
      const int p = por[r];
      for (int t = 0; t < len[p]; ++t) A_dense[(size_t)r * n + col[(size_t)p * cap + t]] = val[(size_t)p * cap + t];
    }
  }
  if (part_of_row) std::copy(por.begin(), por.end(), part_of_row);
  if (orb_of_col) std::copy(ooc.begin(), ooc.end(), orb_of_col);
  return VMC_OK;
}

extern "C" vmc_status vmc_get_factors(vmc_ctx* ctx, int walker, double* L_dense, double* U_dense, int* perm) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  int set = 0;
  if (ctx->pair) {
    CK(cudaMemcpyAsync(&set, &ctx->dCtl[walker].active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "factor set");
    CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  }
  const Walker& W = set ? ctx->hw1[walker] : ctx->hw[walker];
  const int n = W.n, c = W.capLU;
  std::vector<int> lc((size_t)n * c), ll(n), uc((size_t)n * c), ul(n), pm(n);
  std::vector<double> lv((size_t)n * c), uv((size_t)n * c), dv(n);
  CK(d2h(lc.data(), W.l_col, lc.size(), ctx->stream), "factors");
  CK(d2h(lv.data(), W.l_val64, lv.size(), ctx->stream), "factors");
  CK(d2h(ll.data(), W.l_len, ll.size(), ctx->stream), "factors");
  CK(d2h(uc.data(), W.u_col, uc.size(), ctx->stream), "factors");
  CK(d2h(uv.data(), W.u_val64, uv.size(), ctx->stream), "factors");
  CK(d2h(ul.data(), W.u_len, ul.size(), ctx->stream), "factors");
  CK(d2h(dv.data(), W.u_dinv64, dv.size(), ctx->stream), "factors");
  CK(d2h(pm.data(), W.perm, pm.size(), ctx->stream), "factors");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  if (L_dense) {
    std::fill(L_dense, L_dense + (size_t)n * n, 0.0);
    for (int r = 0; r < n; ++r) {
      L_dense[(size_t)r * n + r] = 1.0;
      for (int t = 0; t < ll[r]; ++t) L_dense[(size_t)r * n + lc[(size_t)r * c + t]] = lv[(size_t)r * c + t];
    }
  }
  if (U_dense) {
    std::fill(U_dense, U_dense + (size_t)n * n, 0.0);
    for (int r = 0; r < n; ++r) {
      U_dense[(size_t)r * n + r] = 1.0 / dv[r];
      for (int t = 0; t < ul[r]; ++t) U_dense[(size_t)r * n + uc[(size_t)r * c + t]] = uv[(size_t)r * c + t];
    }
  }
  if (perm) std::copy(pm.begin(), pm.end(), perm);
  return VMC_OK;
}

extern "C" vmc_status vmc_apply_preconditioner(vmc_ctx* ctx, int walker, const double* v, double* z) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || !v || !z || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  const Walker& W = ctx->hw[walker];
  CK(cudaMemcpyAsync(W.r64, v, sizeof(double) * W.n, cudaMemcpyHostToDevice, ctx->stream), "vector");
  CK(launch_apply_precond(cfg(ctx), ctx->dW, walker, ctx->P), "precond kernel");
  CK(cudaMemcpyAsync(z, W.x64, sizeof(double) * W.n, cudaMemcpyDeviceToHost, ctx->stream), "vector");
  CK(cudaStreamSynchronize(ctx->stream), "synchronize");
  ctx->pending[walker] = 0;
  return VMC_OK;
}

extern "C" vmc_status vmc_refactor(vmc_ctx* ctx, int walker, int reorder) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || walker < 0 || walker >= ctx->nw) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  CK(launch_refactor(cfg(ctx), ctx->dW, walker, ctx->P, reorder), "refactor kernel");
  ctx->pending[walker] = 0;
  return check_walker_status(ctx);
}

extern "C" vmc_status vmc_kernel_bench(vmc_ctx* ctx, int which, int reps) {
  if (ctx && ctx->dense) return fail(ctx, VMC_ERR_INVALID, "not available with the dense engine");
  if (!ctx || which < 0 || which > 2 || reps < 1) return fail(ctx, VMC_ERR_INVALID, "bad arguments");
  if (!ctx->ready) return fail(ctx, VMC_ERR_STATE, "positions not set");
  CK(launch_bench(cfg(ctx), ctx->dW, ctx->nw, ctx->P, which, reps), "bench kernel");
  for (int w = 0; w < ctx->nw; ++w) ctx->pending[w] = 0;
  return VMC_OK;
}

extern "C" vmc_status vmc_check_wait_timeout(vmc_ctx* ctx) {
  if (!ctx) return VMC_ERR_INVALID;
  int* d = nullptr;
  int h = -1;
  CK(cudaMalloc((void**)&d, sizeof(int)), "alloc");
  cudaError_t e = launch_wait_timeout(d, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "wait-timeout kernel");
  if (h != ST_TIMEOUT) return fail(ctx, VMC_ERR_STATE, "bounded wait did not report a timeout");
  return fail(ctx, VMC_ERR_TIMEOUT, "device wait gave up after its time limit (expected)");
}

extern "C" vmc_status vmc_philox_device(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
  if (!ctr || !key || !out || n <= 0) return VMC_ERR_INVALID;
  uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
  vmc_status st = VMC_OK;
  if (cudaMalloc((void**)&dc, sizeof(uint32_t) * 4 * n) != cudaSuccess ||
      cudaMalloc((void**)&dk, sizeof(uint32_t) * 2) != cudaSuccess ||
      cudaMalloc((void**)&dout, sizeof(uint32_t) * 4 * n) != cudaSuccess) {
    st = VMC_ERR_OOM;
  } else if (cudaMemcpy(dc, ctr, sizeof(uint32_t) * 4 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(dk, key, sizeof(uint32_t) * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
             launch_philox(dc, dk, dout, n, 0) != cudaSuccess ||
             cudaMemcpy(out, dout, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    st = VMC_ERR_CUDA;
  }
  if (dc) cudaFree(dc);
  if (dk) cudaFree(dk);
  if (dout) cudaFree(dout);
  return st;
}

// ---- autotuner ---------------------------------------------------------------------
static vmc_status tune_trial(const vmc_system* systems, int nw, const vmc_solver_params& p, const uint64_t* seeds,
                             double jitter, const double* xyz, int64_t sweep0, double sigma, int steps, void* stream,
                             double* rate, int* lag, int* mu) {
  vmc_ctx* c = nullptr;
  *rate = 0.0;
  *lag = 0;
  *mu = p.max_updates;
  vmc_status st = vmc_create(systems, nw, &p, stream, &c);
  auto start = [&]() -> vmc_status {
    if (!xyz) return vmc_init_positions(c, seeds, jitter);
    vmc_status s2 = vmc_set_positions_all(c, xyz);
    if (s2 == VMC_OK) s2 = vmc_set_sweep_count(c, sweep0);
    return s2;
  };
  if (st == VMC_OK) {
    if (cudaMemcpyAsync(c->d_seeds, seeds, sizeof(uint64_t) * nw, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      st = VMC_ERR_CUDA;
    else
      st = start();
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == VMC_OK) {
    *lag = c->P.af_lag;
    *mu = c->P.max_updates;
    c->P.step_limit = steps;
    long long moves = 0;
    for (int w = 0; w < nw; ++w) moves += std::min(c->hw[w].n, steps);
    // the persistent engine makes the trial's moves as a budgeted advance (the batch's
    // throughput); the others a partial sweep of `steps` moves per walker
    const bool budget = p.engine == VMC_ENGINE_PERSISTENT;
    auto trial = [&]() -> vmc_status {
      if (budget) {
        c->P.step_limit = 0;
        return vmc_advance_async(c, moves, sigma, c->d_seeds);
      }
      return enqueue_sweeps(c, 1, sigma, c->d_seeds, nullptr, nullptr);
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = VMC_ERR_CUDA;
    if (st == VMC_OK) st = trial();  // untimed
    if (st == VMC_OK && xyz) st = start();  // the timed trial from the same state
    if (st == VMC_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = VMC_ERR_CUDA;
    if (st == VMC_OK) st = trial();  // timed
    if (st == VMC_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) st = VMC_ERR_CUDA;
    if (st == VMC_OK) st = check_walker_status(c);
    float ms = 0.0f;
    if (st == VMC_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f) *rate = moves / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (c) vmc_destroy(c);
  return st;
}

extern "C" vmc_status vmc_autotune_state(const vmc_system* systems, int n_walkers, vmc_solver_params* params,
                                         const uint64_t* seeds, double jitter, const double* xyz, int64_t sweep0,
                                         double sigma, int steps, vmc_tune_trial* trials, int max_trials,
                                         int* n_trials, void* stream) {
  if (n_trials) *n_trials = 0;
  if (!systems || !params || !seeds || n_walkers <= 0 || steps <= 0 || !(sigma >= 0.0) || !(jitter >= 0.0) ||
      sweep0 < 0 || (trials && max_trials < 0) || params->engine == VMC_ENGINE_DENSE_SM)
    return VMC_ERR_INVALID;
  struct Cand { int engine, threads, mu, lag, lfil, group; };
  std::vector<vmc_tune_trial> done;
  vmc_status first_err = VMC_OK;
  auto run = [&](const Cand& cd) -> double {
    vmc_solver_params p = *params;
    p.engine = cd.engine;
    p.block_threads = cd.threads;
    p.max_updates = cd.mu;
    p.refactor_lag = cd.lag;
    p.lfil_extra = cd.lfil;
    p.trisolve_group = cd.group;
    double rate = 0.0;
    int lag = 0, mu = cd.mu;
    const vmc_status st = tune_trial(systems, n_walkers, p, seeds, jitter, xyz, sweep0, sigma, steps, stream, &rate,
                                     &lag, &mu);
    if (st != VMC_OK && first_err == VMC_OK) first_err = st;
    vmc_tune_trial t{cd.engine, cd.threads, mu, lag, st == VMC_OK ? rate : 0.0, (int)st, cd.lfil, cd.group};
    done.push_back(t);
    return st == VMC_OK ? rate : 0.0;
  };
  // phase 1: the ILUTP fill limit (it decides how often the controller must reorder, which
  // dominates the cost of every other choice) with the default mapping
  const int mu0 = params->max_updates;
  double best = -1.0;
  Cand bc{VMC_ENGINE_PERSISTENT, 256, mu0, -1, params->lfil_extra, params->trisolve_group};
  for (int lf : {-1, 16, 32, 48}) {
    Cand cd = bc;
    cd.lfil = lf;
    const double r = run(cd);
    if (r > best) { best = r; bc = cd; }
  }
  // phase 2: mapping x CTA size at that fill limit
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool pairs_fit = auto_pairs_fit(systems, n_walkers, nsm) && (mu0 < 0 || mu0 >= 2);  // refactor_lag = -1's rule
  const Cand b1 = bc;
  for (int threads : {128, 256}) {
    const Cand cands[3] = {{VMC_ENGINE_PERSISTENT, threads, mu0, -1, b1.lfil, b1.group},
                           {VMC_ENGINE_PERSISTENT, threads, mu0, 0, b1.lfil, b1.group},
                           {VMC_ENGINE_STEP, threads, mu0, 0, b1.lfil, b1.group}};
    for (const Cand& cd : cands) {
      if (cd.lag == -1 && (!pairs_fit || threads == 256)) continue;  // (256, -1) was phase 1's trial
      if (cd.lag == 0 && cd.engine == VMC_ENGINE_PERSISTENT && threads == 256 && !pairs_fit) continue;
      const double r = run(cd);
      if (r > best) { best = r; bc = cd; }
    }
  }
  {
    // the record of the best trial holds the lag and chain length it ran with
    for (const vmc_tune_trial& t : done)
      if (t.status == VMC_OK && t.ratios_per_s == best) { bc.lag = t.refactor_lag; bc.mu = t.max_updates; }
  }
  // phase 3: chain length for the best mapping
  const int mu_best = bc.mu;
  for (int mu : {32, 64, 128}) {
    if (mu == mu_best || mu > kMaxUpd) continue;
    Cand cd = bc;
    cd.mu = mu;
    if (bc.lag > 0) cd.lag = -1;  // background lag follows the chain length (mu / 2)
    const double r = run(cd);
    if (r > best) { best = r; bc = cd; bc.lag = done.back().refactor_lag; }
  }
  // phase 4: grouped or level-by-level triangular solves (grouping trades synchronisation
  // for work: it wins where a walker's solve is latency-bound, loses where two walker CTAs
  // share an SM and the work counts)
  {
    Cand cd = bc;
    cd.group = bc.group > 1 ? 1 : 8;
    if (bc.lag > 0) cd.lag = -1;
    const double r = run(cd);
    if (r > best) { best = r; bc = cd; bc.lag = done.back().refactor_lag; }
  }
  if (trials)
    for (int i = 0; i < (int)done.size() && i < max_trials; ++i) trials[i] = done[i];
  if (n_trials) *n_trials = (int)done.size();
  if (best <= 0.0) return first_err != VMC_OK ? first_err : VMC_ERR_INVALID;
  params->engine = bc.engine;
  params->block_threads = bc.threads;
  params->max_updates = bc.mu;
  params->refactor_lag = bc.lag;
  params->lfil_extra = bc.lfil;
  params->trisolve_group = bc.group;
  return VMC_OK;
}

extern "C" vmc_status vmc_autotune(const vmc_system* systems, int n_walkers, vmc_solver_params* params,
                                   const uint64_t* seeds, double jitter, double sigma, int steps,
                                   vmc_tune_trial* trials, int max_trials, int* n_trials, void* stream) {
  return vmc_autotune_state(systems, n_walkers, params, seeds, jitter, nullptr, 0, sigma, steps, trials, max_trials,
                            n_trials, stream);
}
