// vmc_internal.h -- declarations shared by the kernel translation unit and the C ABI
// translation unit (host-side launchers and the layout helpers).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "vmc_device.cuh"

namespace vmc {

struct LaunchCfg {
  cudaStream_t stream;
  int threads;
  bool fp64;
  size_t smem;  // dynamic shared memory per walker CTA
};
// static shared memory of the walker kernels (bytes)
int kernel_static_smem(bool fp64);

cudaError_t launch_sweep(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int n_sweeps,
                         long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc, double* ratio);
// Persistent sweeps with a factor CTA per walker (cluster of 2); see k_sweep_pair.
cudaError_t launch_sweep_pair(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P,
                              int n_sweeps, long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc,
                              double* ratio, int launch_id);
// sweep_dev: nullptr, or a device scalar holding the sweep index (graph replays; then
// sweep0 is ignored)
cudaError_t launch_step(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int q,
                        int n_sweeps, int s_local, long long sweep0, double sigma, const uint64_t* seeds,
                        uint8_t* acc, double* ratio, const long long* sweep_dev = nullptr);
cudaError_t launch_next_sweep(long long* sweep_dev, cudaStream_t s);
cudaError_t launch_set_sweep(long long* sweep_dev, long long v, cudaStream_t s);
// Sets the step kernels' shared-memory attribute (before a graph capture).
cudaError_t prepare_step_kernels(const LaunchCfg& L);
// want_grad: also the gradient and Laplacian at r (Ctl::pend_grad, pend_lap)
cudaError_t launch_ratio(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int k, const double r[3],
                         int want_grad = 0);
cudaError_t launch_accept(const LaunchCfg& L, const Walker* W, int wi, const Params& P);
// Kinetic energy of every walker into out[0 .. nwalk) (device).
cudaError_t launch_kinetic(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, double* out);
cudaError_t launch_init_positions(const LaunchCfg& L, const Walker* W, int nwalk, const uint64_t* seeds, double jitter);
cudaError_t launch_setup(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P);
cudaError_t launch_refactor(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int reorder);
cudaError_t launch_apply_precond(const LaunchCfg& L, const Walker* W, int wi, const Params& P);
cudaError_t launch_bench(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, int which, int reps);
cudaError_t launch_dense_setup(const LaunchCfg& L, const Walker* W, int nwalk);
cudaError_t launch_dense_sweep(const LaunchCfg& L, const Walker* W, int nwalk, int n_sweeps, long long sweep0,
                               double sigma, const uint64_t* seeds, uint8_t* acc, double* ratio, int refresh);
cudaError_t launch_wait_timeout(int* status, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, cudaStream_t s);

// Per-precision instantiations (vmc_engine_f64.cu, vmc_engine_f32.cu) behind the
// launchers above.
template <typename T> int kernel_static_smem_T();
template <typename T>
cudaError_t launch_sweep_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int n_sweeps,
                           long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc, double* ratio);
template <typename T>
cudaError_t launch_sweep_pair_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P,
                                int n_sweeps, long long sweep0, double sigma, const uint64_t* seeds, uint8_t* acc,
                                double* ratio, int launch_id);
template <typename T> cudaError_t prepare_step_kernels_T(const LaunchCfg& L);
template <typename T>
cudaError_t launch_step_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P, int q,
                          int n_sweeps, int s_local, long long sweep0, double sigma, const uint64_t* seeds,
                          uint8_t* acc, double* ratio, const long long* sweep_dev);
template <typename T>
cudaError_t launch_ratio_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int k, const double r[3],
                           int want_grad);
template <typename T>
cudaError_t launch_kinetic_T(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, double* out);
template <typename T> cudaError_t launch_accept_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P);
template <typename T>
cudaError_t launch_setup_T(const LaunchCfg& L, const Walker* W, int walker0, int nwalk, const Params& P);
template <typename T>
cudaError_t launch_refactor_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P, int reorder);
template <typename T> cudaError_t launch_apply_precond_T(const LaunchCfg& L, const Walker* W, int wi, const Params& P);
template <typename T>
cudaError_t launch_bench_T(const LaunchCfg& L, const Walker* W, int nwalk, const Params& P, int which, int reps);

// Shared-memory plan of a walker CTA: two solve vectors (2 ybytes) in shared memory
// when they fit next to four ring slots and allow_sf (synchronisation-free triangular
// solves), else one when it fits next to two slots, else none; then 16 KB slots when at
// least four fit, else 8 KB.  Fills tri_sf, y_half, y_smem, y_bytes, ring_slots,
// slot_bytes, dsm_bytes.
void plan_smem(int ybytes, int budget, Params& P, bool allow_sf);
// Entries of an expanded row of the grouped triangular solves (a multiple of 4).
int expanded_row_cap(int capLU, int row_cap);
bool rows_fit_slot(int cap, int lfil_extra, int row_cap);

// host-side geometry and layout
struct Layout {
  int n, per, cap;
  std::vector<double> Z;       // n*3
  std::vector<int> col_of_orb;  // n
  std::vector<int> orb_of_col;  // n
};
// Returns 0, or a nonzero code with a message on invalid parameters.
int make_layout(int K, int lattice, double a, double r_c, Layout& out, const char** why);

}  // namespace vmc
