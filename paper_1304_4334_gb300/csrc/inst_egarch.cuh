// Instantiation helpers: one translation unit per (precision, K) keeps each
// compile short and lets the build run them in parallel.
#pragma once

#include "kernels.cuh"

namespace smc {

inline int mutate_grid(int P, int threads = kMutThreads) { return (P + threads - 1) / threads; }

// One particle per thread; threads = a multiple of 32 up to kMutMaxThreads (the caller checks).
template <template <int, int> class Pol, int K>
cudaError_t launch_mutate_k(const MutateArgs& a, int threads, cudaStream_t s)
{
    const int g = mutate_grid(a.P, threads);
    if (a.qmean) {   // independent sampler
        switch (a.m.I) {
        case 1: k_mutate<Pol<K, 1>, true><<<g, threads, 0, s>>>(a); break;
        case 2: k_mutate<Pol<K, 2>, true><<<g, threads, 0, s>>>(a); break;
        case 3: k_mutate<Pol<K, 3>, true><<<g, threads, 0, s>>>(a); break;
        case 4: k_mutate<Pol<K, 4>, true><<<g, threads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    void (*k)(MutateArgs) = nullptr;
    switch (a.m.I) {
    case 1: k = k_mutate<Pol<K, 1>>; break;
    case 2: k = k_mutate<Pol<K, 2>>; break;
    case 3: k = k_mutate<Pol<K, 3>>; break;
    case 4: k = k_mutate<Pol<K, 4>>; break;
    default: return cudaErrorInvalidValue;
    }
    if (a.dependent) return pdl_launch(k, g, threads, 0, s, a);
    k<<<g, threads, 0, s>>>(a);
    return cudaGetLastError();
}

// ppt = particles per thread (1 or 2; 2 only for the FP32 policy)
template <int K>
cudaError_t launch_mutate_x2_k(const MutateArgs& a, int threads, cudaStream_t s)
{
    const int g = (a.P + 2 * threads - 1) / (2 * threads);
    void (*k)(MutateArgs) = nullptr;
    switch (a.m.I) {
    case 1: k = k_mutate_x2<K, 1>; break;
    case 2: k = k_mutate_x2<K, 2>; break;
    case 3: k = k_mutate_x2<K, 3>; break;
    case 4: k = k_mutate_x2<K, 4>; break;
    default: return cudaErrorInvalidValue;
    }
    if (a.dependent) return pdl_launch(k, g, threads, 0, s, a);
    k<<<g, threads, 0, s>>>(a);
    return cudaGetLastError();
}

template <template <int, int> class Pol, int K>
cudaError_t launch_loglik_k(const LoglikArgs& a, cudaStream_t s)
{
    const int g = mutate_grid(a.P);
    switch (a.m.I) {
    case 1: k_loglik<Pol<K, 1>><<<g, kMutThreads, 0, s>>>(a); break;
    case 2: k_loglik<Pol<K, 2>><<<g, kMutThreads, 0, s>>>(a); break;
    case 3: k_loglik<Pol<K, 3>><<<g, kMutThreads, 0, s>>>(a); break;
    case 4: k_loglik<Pol<K, 4>><<<g, kMutThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <template <int, int> class Pol, int K>
cudaError_t launch_cdata_k(const CdataArgs& a, cudaStream_t s)
{
    const int g = mutate_grid(a.P);
    switch (a.m.I) {
    case 1: k_cdata<Pol<K, 1>><<<g, kMutThreads, 0, s>>>(a); break;
    case 2: k_cdata<Pol<K, 2>><<<g, kMutThreads, 0, s>>>(a); break;
    case 3: k_cdata<Pol<K, 3>><<<g, kMutThreads, 0, s>>>(a); break;
    case 4: k_cdata<Pol<K, 4>><<<g, kMutThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace smc

// POL: the mutation kernels' policy; POL_EVAL: the stand-alone likelihood's
// and the data-tempering C phase's.
#define SMC_INSTANTIATE_EGARCH(TAG, POL, POL_EVAL, K)                                           \
    namespace smc {                                                                             \
    cudaError_t launch_mutate_##TAG##_k##K(const MutateArgs& a, int threads, cudaStream_t s)    \
    {                                                                                           \
        return launch_mutate_k<POL, K>(a, threads, s);                                          \
    }                                                                                           \
    cudaError_t launch_loglik_##TAG##_k##K(const LoglikArgs& a, cudaStream_t s)                 \
    {                                                                                           \
        return launch_loglik_k<POL_EVAL, K>(a, s);                                              \
    }                                                                                           \
    cudaError_t launch_cdata_##TAG##_k##K(const CdataArgs& a, cudaStream_t s)                   \
    {                                                                                           \
        return launch_cdata_k<POL_EVAL, K>(a, s);                                               \
    }                                                                                           \
    }
