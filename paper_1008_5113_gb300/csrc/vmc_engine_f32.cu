// vmc_engine_f32.cu -- the engine's kernels and launchers in the
// FP32 (mixed-precision) working precision.
#include "vmc_engine_impl.cuh"

namespace vmc {

template int kernel_static_smem_T<float>();
template cudaError_t launch_sweep_T<float>(const LaunchCfg&, const Walker*, int, int, const Params&, int, long long,
                                         double, const uint64_t*, uint8_t*, double*);
template cudaError_t launch_sweep_pair_T<float>(const LaunchCfg&, const Walker*, int, int, const Params&, int,
                                              long long, double, const uint64_t*, uint8_t*, double*, int);
template cudaError_t prepare_step_kernels_T<float>(const LaunchCfg&);
template cudaError_t launch_step_T<float>(const LaunchCfg&, const Walker*, int, int, const Params&, int, int, int,
                                        long long, double, const uint64_t*, uint8_t*, double*, const long long*);
template cudaError_t launch_ratio_T<float>(const LaunchCfg&, const Walker*, int, const Params&, int, const double*,
                                         int);
template cudaError_t launch_kinetic_T<float>(const LaunchCfg&, const Walker*, int, const Params&, double*);
template cudaError_t launch_accept_T<float>(const LaunchCfg&, const Walker*, int, const Params&);
template cudaError_t launch_setup_T<float>(const LaunchCfg&, const Walker*, int, int, const Params&);
template cudaError_t launch_refactor_T<float>(const LaunchCfg&, const Walker*, int, const Params&, int);
template cudaError_t launch_apply_precond_T<float>(const LaunchCfg&, const Walker*, int, const Params&);
template cudaError_t launch_bench_T<float>(const LaunchCfg&, const Walker*, int, const Params&, int, int);

}  // namespace vmc
