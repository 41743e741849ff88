// Dispatch of the gradient and MALA kernels over model, precision and K.
#include "mala.cuh"

namespace smc {

void count_launch();
#define SMC_DECL_MALA(TAG, K)                                                 \
    cudaError_t launch_grad_##TAG##_k##K(const GradArgs& a, cudaStream_t s); \
    cudaError_t launch_mala_##TAG##_k##K(const MalaArgs& a, cudaStream_t s);
SMC_DECL_MALA(f32, 1)
SMC_DECL_MALA(f32, 2)
SMC_DECL_MALA(f32, 3)
SMC_DECL_MALA(f32, 4)
SMC_DECL_MALA(f64, 1)
SMC_DECL_MALA(f64, 2)
SMC_DECL_MALA(f64, 3)
SMC_DECL_MALA(f64, 4)

cudaError_t launch_loglik_grad(const GradArgs& a, int precision, cudaStream_t s)
{
    count_launch();
    if (a.m.kind == 1) return launch_grad_t<GradLinreg>(a, s);
    if (precision == 1) {
        switch (a.m.K) {
        case 1: return launch_grad_f32_k1(a, s);
        case 2: return launch_grad_f32_k2(a, s);
        case 3: return launch_grad_f32_k3(a, s);
        case 4: return launch_grad_f32_k4(a, s);
        }
    } else {
        switch (a.m.K) {
        case 1: return launch_grad_f64_k1(a, s);
        case 2: return launch_grad_f64_k2(a, s);
        case 3: return launch_grad_f64_k3(a, s);
        case 4: return launch_grad_f64_k4(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mala(const MalaArgs& a, int precision, cudaStream_t s)
{
    count_launch();
    if (a.m.kind == 1) return launch_mala_t<GradLinreg>(a, s);
    if (precision == 1) {
        switch (a.m.K) {
        case 1: return launch_mala_f32_k1(a, s);
        case 2: return launch_mala_f32_k2(a, s);
        case 3: return launch_mala_f32_k3(a, s);
        case 4: return launch_mala_f32_k4(a, s);
        }
    } else {
        switch (a.m.K) {
        case 1: return launch_mala_f64_k1(a, s);
        case 2: return launch_mala_f64_k2(a, s);
        case 3: return launch_mala_f64_k3(a, s);
        case 4: return launch_mala_f64_k4(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace smc
