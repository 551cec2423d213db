// vmc_engine.cu -- the engine's launch entry points: dispatch to the FP64 or FP32
// instantiation of the templated kernels (vmc_engine_impl.cuh), and the small kernels
// that do not depend on the working precision (start positions, sweep index, the
// bounded-wait check, the device random-number generator).
#include "vmc_internal.h"
#include "vmc_geom.cuh"

namespace vmc {

// r = wrap(Z + jitter * N(0,1)^3), purpose 0, sweep 0.
__global__ void k_init_positions(const Walker* __restrict__ W, const uint64_t* __restrict__ seeds, double jitter) {
  const Walker& w = W[blockIdx.x];
  const uint64_t seed = seeds[blockIdx.x];
  for (int i = threadIdx.x; i < w.n; i += blockDim.x) {
    double z[3];
    normal3(seed, 0u, (uint32_t)i, 0u, z);
    for (int d = 0; d < 3; ++d) w.R[3 * i + d] = wrap_box(__dadd_rn(w.Z[3 * i + d], __dmul_rn(jitter, z[d])), w.L);
  }
}

// Failure-detection check: wait on an mbarrier phase that nothing completes, with
// the same bounded wait the solver uses; records ST_TIMEOUT when it gives up.
__global__ void k_wait_timeout(int* status) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0u);  // phase 0 never completes: no arrival is made
  if (threadIdx.x == 0) *status = ok ? ST_OK : ST_TIMEOUT;
}

__global__ void k_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  uint32_t k[2] = {key[0], key[1]};
  uint32_t o[4];
  philox4x32_10(c, k, o);
  for (int j = 0; j < 4; ++j) out[4 * i + j] = o[j];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int kernel_static_smem(bool fp64) { return fp64 ? kernel_static_smem_T<double>() : kernel_static_smem_T<float>(); }

cudaError_t launch_sweep(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int n_sweeps,
                         long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc, double* ratio) {
  return L.fp64 ? launch_sweep_T<double>(L, W, walker0, nwalk, P, n_sweeps, sweep0, sigma, seeds, acc, ratio)
                : launch_sweep_T<float>(L, W, walker0, nwalk, P, n_sweeps, sweep0, sigma, seeds, acc, ratio);
}
cudaError_t launch_sweep_pair(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P,
                              int n_sweeps, long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc,
                              double* ratio, int launch_id) {
  return L.fp64 ? launch_sweep_pair_T<double>(L, W, walker0, nwalk, P, n_sweeps, sweep0, sigma, seeds, acc, ratio,
                                              launch_id)
                : launch_sweep_pair_T<float>(L, W, walker0, nwalk, P, n_sweeps, sweep0, sigma, seeds, acc, ratio,
                                             launch_id);
}
// Advance / set the device-side sweep index of the replayed sweep graphs.
__global__ void k_next_sweep(long long* sweep_dev) { *sweep_dev += 1; }
__global__ void k_set_sweep(long long* sweep_dev, long long v) { *sweep_dev = v; }
cudaError_t launch_set_sweep(long long* sweep_dev, long long v, cudaStream_t s) {
  k_set_sweep<<<1, 1, 0, s>>>(sweep_dev, v);
  return cudaGetLastError();
}
cudaError_t launch_next_sweep(long long* sweep_dev, cudaStream_t s) {
  k_next_sweep<<<1, 1, 0, s>>>(sweep_dev);
  return cudaGetLastError();
}
cudaError_t prepare_step_kernels(const LaunchCfg& L) {
  return L.fp64 ? prepare_step_kernels_T<double>(L) : prepare_step_kernels_T<float>(L);
}
cudaError_t launch_step(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int q,
                        int n_sweeps, int s_local, long long sweep0, double sigma, const uint64_t* seeds,
                        uint8_t* acc, double* ratio, const long long* sweep_dev) {
  return L.fp64 ? launch_step_T<double>(L, W, walker0, nwalk, P, q, n_sweeps, s_local, sweep0, sigma, seeds, acc,
                                        ratio, sweep_dev)
                : launch_step_T<float>(L, W, walker0, nwalk, P, q, n_sweeps, s_local, sweep0, sigma, seeds, acc,
                                       ratio, sweep_dev);
}
cudaError_t launch_ratio(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int k, const double r[3],
                         int want_grad) {
  return L.fp64 ? launch_ratio_T<double>(L, W, wi, P, k, r, want_grad)
                : launch_ratio_T<float>(L, W, wi, P, k, r, want_grad);
}
cudaError_t launch_kinetic(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, double* out) {
  return L.fp64 ? launch_kinetic_T<double>(L, W, nwalk, P, out) : launch_kinetic_T<float>(L, W, nwalk, P, out);
}
cudaError_t launch_accept(const LaunchCfg& L, const Walker* W, int wi, const Params& P) {
  return L.fp64 ? launch_accept_T<double>(L, W, wi, P) : launch_accept_T<float>(L, W, wi, P);
}
cudaError_t launch_init_positions(const LaunchCfg& L, const Walker* W, int nwalk, const uint64_t* seeds, double jitter) {
  k_init_positions<<<nwalk, 256, 0, L.stream>>>(W, seeds, jitter);
  return cudaGetLastError();
}
cudaError_t launch_setup(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P) {
  return L.fp64 ? launch_setup_T<double>(L, W, walker0, nwalk, P) : launch_setup_T<float>(L, W, walker0, nwalk, P);
}
cudaError_t launch_refactor(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int reorder) {
  return L.fp64 ? launch_refactor_T<double>(L, W, wi, P, reorder) : launch_refactor_T<float>(L, W, wi, P, reorder);
}
cudaError_t launch_apply_precond(const LaunchCfg& L, const Walker* W, int wi, const Params& P) {
  return L.fp64 ? launch_apply_precond_T<double>(L, W, wi, P) : launch_apply_precond_T<float>(L, W, wi, P);
}
cudaError_t launch_bench(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, int which, int reps) {
  return L.fp64 ? launch_bench_T<double>(L, W, nwalk, P, which, reps) : launch_bench_T<float>(L, W, nwalk, P, which, reps);
}
cudaError_t launch_wait_timeout(int* status, cudaStream_t s) {
  k_wait_timeout<<<1, 32, 0, s>>>(status);
  return cudaGetLastError();
}
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, cudaStream_t s) {
  k_philox<<<(n + 127) / 128, 128, 0, s>>>(ctr, key, out, n);
  return cudaGetLastError();
}

}  // namespace vmc
