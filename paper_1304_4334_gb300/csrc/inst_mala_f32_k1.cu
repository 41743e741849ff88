// FP32 gradient and MALA kernels, K = 1 volatility factors, I = 1..4.
#include "mala.cuh"
namespace smc {
cudaError_t launch_grad_f32_k1(const GradArgs& a, cudaStream_t s) { return launch_grad_k<float, 1>(a, s); }
cudaError_t launch_mala_f32_k1(const MalaArgs& a, cudaStream_t s) { return launch_mala_k<float, 1>(a, s); }
}  // namespace smc
