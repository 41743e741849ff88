// Conjugate normal linear regression kernels (FP64), the closed-form check model.
#include "inst_egarch.cuh"

namespace smc {

cudaError_t launch_mutate_linreg(const MutateArgs& a, int threads, cudaStream_t s)
{
    if (a.qmean) k_mutate<PolicyLinreg, true><<<mutate_grid(a.P, threads), threads, 0, s>>>(a);
    else k_mutate<PolicyLinreg><<<mutate_grid(a.P, threads), threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_loglik_linreg(const LoglikArgs& a, cudaStream_t s)
{
    k_loglik<PolicyLinreg><<<mutate_grid(a.P), kMutThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cdata_linreg(const CdataArgs& a, cudaStream_t s)
{
    k_cdata<PolicyLinreg><<<mutate_grid(a.P), kMutThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace smc
