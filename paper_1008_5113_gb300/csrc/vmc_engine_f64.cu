// vmc_engine_f64.cu -- the engine's kernels and launchers in the
// FP64 working precision.
#include "vmc_engine_impl.cuh"

namespace vmc {

template int kernel_static_smem_T<double>();
template cudaError_t launch_sweep_T<double>(const LaunchCfg&, const Walker*, int, int, const Params&, int, long long,
                                         double, const uint64_t*, uint8_t*, double*);
template cudaError_t launch_sweep_pair_T<double>(const LaunchCfg&, const Walker*, int, int, const Params&, int,
                                              long long, double, const uint64_t*, uint8_t*, double*, int);
template cudaError_t prepare_step_kernels_T<double>(const LaunchCfg&);
template cudaError_t launch_step_T<double>(const LaunchCfg&, const Walker*, int, int, const Params&, int, int, int,
                                        long long, double, const uint64_t*, uint8_t*, double*, const long long*);
template cudaError_t launch_ratio_T<double>(const LaunchCfg&, const Walker*, int, const Params&, int, const double*,
                                         int);
template cudaError_t launch_kinetic_T<double>(const LaunchCfg&, const Walker*, int, const Params&, double*);
template cudaError_t launch_accept_T<double>(const LaunchCfg&, const Walker*, int, const Params&);
template cudaError_t launch_setup_T<double>(const LaunchCfg&, const Walker*, int, int, const Params&);
template cudaError_t launch_refactor_T<double>(const LaunchCfg&, const Walker*, int, const Params&, int);
template cudaError_t launch_apply_precond_T<double>(const LaunchCfg&, const Walker*, int, const Params&);
template cudaError_t launch_bench_T<double>(const LaunchCfg&, const Walker*, int, const Params&, int, int);

}  // namespace vmc
