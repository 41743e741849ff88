// FP32 EGARCH kernels with K = 3 volatility factors, I = 1..4 mixture components.
#include "inst_egarch.cuh"
SMC_INSTANTIATE_EGARCH(f32, PolicyEgarchF32, PolicyEgarchF32Delta, 3)
namespace smc {
cudaError_t launch_mutate_x2_f32_k3(const MutateArgs& a, int threads, cudaStream_t s)
{
    return launch_mutate_x2_k<3>(a, threads, s);
}
}  // namespace smc
