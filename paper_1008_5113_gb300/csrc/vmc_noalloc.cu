// vmc_noalloc.cu -- vmc_ratio_noalloc: the determinant ratio of one move of one
// walker with no device allocation at all.
//
// Callers that cannot call cudaMalloc: code that runs where allocation is not
// allowed or not wanted -- inside a framework that owns all device memory through
// its own pool and forbids raw allocations, in latency-critical paths where a
// cudaMalloc (which can synchronise the device) is unacceptable, or after an
// application has reserved all free memory for itself.  For them this entry point
// keeps the whole walker workspace (matrix slots, ILUTP factors and their streams,
// Krylov basis, update chain, controller state) in one file-scope device array of
// fixed size, kNoAllocBytes, which every GPU that loads the library holds until
// the process exits.  The caller passes the inputs and the output.
//
// The device address of that array is looked up with cudaGetSymbolAddress on the
// first call made with a device current, and again whenever that device's context
// has changed since (after a cudaDeviceReset the module is loaded anew, possibly at
// another address); the first call on a device should therefore come before any
// stream capture.  Every call reuses
// the same array and overwrites the previous call's contents (the used part is
// cleared at the start of each call), so calls that overlap on the GPU -- on
// different streams or from different host threads -- race and must not be issued.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vmc.h"
#include "vmc_internal.h"

using namespace vmc;

namespace {

constexpr size_t kNoAllocBytes = (size_t)16 << 20;  // 16 MiB of device scratch
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};  // the context the address belongs to
thread_local std::string g_noalloc_error;

// The driver's cuCtxGetCurrent, reached through the runtime (no link against libcuda).
using CtxGetCurrentFn = int (*)(void**);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (CtxGetCurrentFn)f;
  }();
  return fn;
}

// Device address of the scratch array for the current device: looked up on the first
// call with this device current, and again when the device's context has changed.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const CtxGetCurrentFn get = ctx_get_current();
  if (!get) return cudaErrorDeviceUninitialized;
  void* cur = nullptr;
  if (get(&cur) != 0) cur = nullptr;  // null before the runtime has made a context current
  std::lock_guard<std::mutex> lk(g_mu);
  if (!cur || !g_scratch_addr[dev] || g_scratch_ctx[dev] != cur) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // initialises the context if need be
    if (e != cudaSuccess) return e;
    if (get(&cur) != 0 || !cur) return cudaErrorDeviceUninitialized;
    g_scratch_addr[dev] = (unsigned char*)p;
    g_scratch_ctx[dev] = cur;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

struct Off {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t o = off;
    off += count * sizeof(T);
    return o;
  }
};

vmc_status fail(vmc_status s, const std::string& m) {
  g_noalloc_error = m;
  return s;
}

}  // namespace

extern "C" const char* vmc_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" size_t vmc_noalloc_capacity(void) { return kNoAllocBytes; }

extern "C" vmc_status vmc_ratio_noalloc(const vmc_system* sys, const vmc_solver_params* params,
                                        const double* xyz_dev, int k, const double r_new[3], double* ratio_dev,
                                        void* stream) {
  g_noalloc_error.clear();
  if (!sys || !xyz_dev || !r_new || !ratio_dev) return fail(VMC_ERR_INVALID, "null argument");
  vmc_solver_params p;
  if (params) p = *params;
  else vmc_default_params(&p);
  if (p.max_updates < 0) p.max_updates = 128;  // auto: the in-line default
  if (p.gmres_m < 1 || p.gmres_m > kMaxM || p.max_updates > kMaxUpd ||
      (p.precision != VMC_PREC_FP64 && p.precision != VMC_PREC_MIXED && p.precision != VMC_PREC_MIXED_F32ILU) ||
      (p.block_threads != 0 && (p.block_threads < 64 || p.block_threads > kMaxThreads || p.block_threads % 32)) ||
      !(p.drop_tol >= 0.0) || !(p.permtol >= 0.0) || p.max_restarts < 0 || p.trisolve_row_cap < 0 ||
      p.trisolve_row_cap > 480 || p.trisolve_lane_entries < 0 || p.trisolve_lane_entries > 64)
    return fail(VMC_ERR_INVALID, "invalid solver parameters");
  Layout lay;
  const char* why = "";
  if (make_layout(sys->K, sys->lattice, sys->a, sys->r_c, lay, &why)) return fail(VMC_ERR_INVALID, why);
  if (!(sys->kappa > 0.0)) return fail(VMC_ERR_INVALID, "kappa must be positive");
  if (!rows_fit_slot(lay.cap, p.lfil_extra, p.trisolve_row_cap))
    return fail(VMC_ERR_INVALID, "factor rows longer than a stream slot (r_c or lfil_extra too large)");
  const int n = lay.n, cap = lay.cap;
  if (k < 0 || k >= n) return fail(VMC_ERR_INVALID, "particle index out of range");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(r_new[d])) return fail(VMC_ERR_INVALID, "non-finite position");
  const bool fp64 = p.precision == VMC_PREC_FP64;
  const size_t Tsz = fp64 ? sizeof(double) : sizeof(float);
  const int m = p.gmres_m, mu = std::max(1, p.max_updates);
  const int pmax = p.lfil_extra >= 0 ? p.lfil_extra : (cap + 1) / 2;
  const int capLU = (cap + pmax + 2 + 3) / 4 * 4;
  const int exmax = expanded_row_cap(capLU, p.trisolve_row_cap);
  const size_t sbytes = (size_t)n * (256 + 12 * (size_t)std::max(capLU, exmax));

  // carve the walker workspace out of the scratch array
  Off o;
  const size_t oZ = o.take<double>((size_t)n * 3), oCO = o.take<int>(n), oOC = o.take<int>(n);
  const size_t oR = o.take<double>((size_t)n * 3), oRP = o.take<int>(n), oPR = o.take<int>(n);
  const size_t oAc = o.take<int>((size_t)n * cap), oAv = o.take<double>((size_t)n * cap);
  const size_t oAv32 = o.take<float>((size_t)n * cap), oAl = o.take<int>(n);
  const size_t oLc = o.take<int>((size_t)n * capLU), oLv = o.take<double>((size_t)n * capLU);
  const size_t oLs = o.take<unsigned char>(sbytes), oLl = o.take<int>(n);
  const size_t oUc = o.take<int>((size_t)n * capLU), oUv = o.take<double>((size_t)n * capLU);
  const size_t oUs = o.take<unsigned char>(sbytes), oUl = o.take<int>(n), oUd = o.take<double>(n);
  const size_t oCh = o.take<int2>(2 * (size_t)n + 2);
  const size_t oPm = o.take<int>(n), oIp = o.take<int>(n), oLvl = o.take<int>(n), oUvl = o.take<int>(n);
  const size_t oLlp = o.take<int>(n + 1), oLlr = o.take<int>(n), oUlp = o.take<int>(n + 1), oUlr = o.take<int>(n);
  const size_t oCur = o.take<int>(n + 1), oWr = o.take<double>(n), oWp = o.take<int>(n);
  const size_t oGP = o.take<int>(n), oGQ = o.take<int>(n);
  const size_t oUz = o.take<char>((size_t)((mu + 3) / 4 * 4) * n * Tsz), oUuc = o.take<int>((size_t)mu * kMaxU);
  const size_t oUuv = o.take<char>((size_t)mu * kMaxU * Tsz), oUul = o.take<int>(mu);
  const size_t oG = o.take<double>((size_t)kMaxUpd * kMaxUpd);
  const size_t oV = o.take<char>((size_t)(m + 1) * n * Tsz), oZk = o.take<char>((size_t)m * n * Tsz);
  const size_t oTv = o.take<char>((size_t)3 * n * Tsz), oX = o.take<double>(n), oRr = o.take<double>(n);
  const size_t oPac = o.take<int>(cap), oPav = o.take<double>(cap), oPuc = o.take<int>(kMaxU);
  const size_t oPuv = o.take<double>(kMaxU), oMeta = o.take<int4>(n + 1), oLnc = o.take<int>(n + 1);
  const size_t oSeg = o.take<int4>(2 * (size_t)n + 2);
  const size_t oUh = o.take<double2>(n);
  const size_t oExl = o.take<int>(n), oExc = o.take<int>((size_t)n * exmax), oExv = o.take<double>((size_t)n * exmax);
  const size_t oGp = o.take<int>(n + 1);
  const size_t oCtl = o.take<Ctl>(1), oW = o.take<Walker>(1);
  const size_t used = o.off;
  if (used > kNoAllocBytes)
    return fail(VMC_ERR_CAPACITY, "system too large for the no-allocation scratch: needs " + std::to_string(used) +
                                      " bytes, the fixed maximum is " + std::to_string(kNoAllocBytes));

  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail(VMC_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;

  Walker W;
  std::memset(&W, 0, sizeof(W));
  W.n = n; W.K = sys->K; W.lattice = sys->lattice; W.cap = cap; W.capLU = capLU; W.m = m; W.mu = mu; W.mu4 = (mu + 3) / 4 * 4; W.per = lay.per;
  W.a = sys->a; W.kappa = sys->kappa; W.rc = sys->r_c; W.rc2 = sys->r_c * sys->r_c; W.L = sys->K * sys->a;
  W.Z = (const double*)(base + oZ); W.col_of_orb = (const int*)(base + oCO); W.orb_of_col = (const int*)(base + oOC);
  W.R = (double*)(base + oR); W.row_of_part = (int*)(base + oRP); W.part_of_row = (int*)(base + oPR);
  W.a_col = (int*)(base + oAc); W.a_val = (double*)(base + oAv); W.a_val32 = (float*)(base + oAv32);
  W.a_len = (int*)(base + oAl);
  W.l_col = (int*)(base + oLc); W.l_val64 = (double*)(base + oLv); W.lstream = base + oLs; W.l_len = (int*)(base + oLl);
  W.u_col = (int*)(base + oUc); W.u_val64 = (double*)(base + oUv); W.ustream = base + oUs; W.u_len = (int*)(base + oUl);
  W.u_dinv64 = (double*)(base + oUd);
  W.u_head = (double2*)(base + oUh);
  W.exmax = exmax;
  W.ex_len = (int*)(base + oExl); W.ex_col = (int*)(base + oExc); W.ex_val = (double*)(base + oExv);
  W.gptr = (int*)(base + oGp);
  W.lchunk = (int2*)(base + oCh); W.uchunk = W.lchunk + (n + 1);
  W.perm = (int*)(base + oPm); W.iperm = (int*)(base + oIp); W.lev_l = (int*)(base + oLvl); W.lev_u = (int*)(base + oUvl);
  W.l_lvl_ptr = (int*)(base + oLlp); W.l_lvl_rows = (int*)(base + oLlr);
  W.u_lvl_ptr = (int*)(base + oUlp); W.u_lvl_rows = (int*)(base + oUlr); W.lvl_cur = (int*)(base + oCur);
  W.wrow = (double*)(base + oWr); W.wpos = (int*)(base + oWp); W.gP = (int*)(base + oGP); W.gQ = (int*)(base + oGQ);
  W.upd_z = base + oUz; W.upd_ucol = (int*)(base + oUuc); W.upd_uval = base + oUuv; W.upd_ulen = (int*)(base + oUul);
  W.upd_G = (double*)(base + oG);
  W.V = base + oV; W.Zk = base + oZk; W.tv = base + oTv; W.x64 = (double*)(base + oX); W.r64 = (double*)(base + oRr);
  W.pend_acol = (int*)(base + oPac); W.pend_aval = (double*)(base + oPav);
  W.pend_ucol = (int*)(base + oPuc); W.pend_uval = (double*)(base + oPuv);
  W.chunk_meta = (int4*)(base + oMeta); W.lvl_nchunk = (int*)(base + oLnc);
  W.seg_meta = (int4*)(base + oSeg);
  W.ctl = (Ctl*)(base + oCtl);
  W.log_base = 0;
  Walker* dW = (Walker*)(base + oW);

  Params P{};
  P.drop_tol = p.drop_tol; P.permtol = p.permtol; P.lfil_extra = p.lfil_extra; P.m = m;
  P.max_restarts = p.max_restarts; P.max_updates = p.max_updates;
  P.inner_rtol = p.inner_rtol > 0.0 ? p.inner_rtol : (fp64 ? 1e-10 : 1e-5);
  P.ratio_tol = p.ratio_tol > 0.0 ? p.ratio_tol : 1e-12;
  P.ilu64 = p.precision != VMC_PREC_MIXED_F32ILU;
  P.N_max = p.N_max; P.slow_factor = p.slow_factor;
  P.trig_rtol = p.trigger_rtol > 0.0 ? p.trigger_rtol : 1e-6;
  P.trig_its = p.trigger_its > 0 ? p.trigger_its : 40;
  P.ilu_variant = (p.ilutp_variant >= 0 && p.ilutp_variant <= 2) ? p.ilutp_variant : 0;
  P.warp_rows = std::min(std::max(p.trisolve_warp_rows, 0), 32);
  P.tri_group = p.trisolve == 1 ? 1 : std::min(std::max(p.trisolve_group, 1), 64);
  P.lane_entries = p.trisolve_lane_entries > 0 ? std::min(p.trisolve_lane_entries, 64) : (fp64 ? 8 : 2);
  P.step_limit = 0;
  // shared-memory plan for a single walker CTA
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int stat = kernel_static_smem(fp64);
  if (optin <= 0 || stat <= 0) return fail(VMC_ERR_CUDA, "no usable CUDA device");
  const int ybytes1 = (int)(((size_t)n * Tsz + 127) / 128 * 128);
  const int ybytes = P.tri_group > 1 ? (int)(((size_t)2 * n * Tsz + 127) / 128 * 128) : ybytes1;
  const int budget = optin - stat;
  plan_smem(ybytes, budget, P, p.trisolve == 1);
  if (!P.y_smem && ybytes != ybytes1) plan_smem(ybytes1, budget, P, p.trisolve == 1);
  const LaunchCfg L{s, p.block_threads ? p.block_threads : 256, fp64, (size_t)P.dsm_bytes};

  // clear the part of the scratch this call uses, then fill the inputs
  e = cudaMemsetAsync(base, 0, used, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + oZ, lay.Z.data(), sizeof(double) * lay.Z.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + oCO, lay.col_of_orb.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + oOC, lay.orb_of_col.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + oR, xyz_dev, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dW, &W, sizeof(Walker), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(VMC_ERR_CUDA, std::string("scratch fill: ") + cudaGetErrorString(e));
  // the positions are taken as given (inside the box); setup = rows, reorder, ILUTP
  e = launch_setup(L, dW, 0, 1, P);
  if (e == cudaSuccess) e = launch_ratio(L, dW, 0, P, k, r_new);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ratio_dev, &W.ctl->pend_ratio, sizeof(double), cudaMemcpyDeviceToDevice, s);
  int st[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st[0], &W.ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st[1], &W.ctl->pend_valid, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(VMC_ERR_CUDA, std::string("ratio: ") + cudaGetErrorString(e));
  if (st[0] != ST_OK) return fail((vmc_status)st[0], "walker failed with status " + std::to_string(st[0]));
  if (!st[1]) return fail(VMC_ERR_NOCONV, "solve did not converge");
  return VMC_OK;
}
