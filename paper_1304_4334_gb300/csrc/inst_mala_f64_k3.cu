// FP64 gradient and MALA kernels, K = 3 volatility factors, I = 1..4.
#include "mala.cuh"
namespace smc {
cudaError_t launch_grad_f64_k3(const GradArgs& a, cudaStream_t s) { return launch_grad_k<double, 3>(a, s); }
cudaError_t launch_mala_f64_k3(const MalaArgs& a, cudaStream_t s) { return launch_mala_k<double, 3>(a, s); }
}  // namespace smc
