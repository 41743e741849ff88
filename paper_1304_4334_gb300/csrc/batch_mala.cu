// Batched MALA: the persistent M-phase kernel of the batched driver for runs
// whose mutation is the Langevin proposal (FP32 EGARCH, power tempering).
//
// Like the random-walk batch kernel, persistent blocks pull work items
// (dataset, tile of particles) from one queue ordered by decreasing cost, so
// that datasets of very different length and model share the GPU.  Each
// particle runs exactly the single-run MALA step (mala_particle): proposal with
// the drift (1/2) L L' g from its stored gradient, log likelihood and gradient
// of the proposal by the forward recursion and the hand-written reverse sweep,
// and the Metropolis-Hastings ratio with the reverse proposal density.  Every
// thread keeps the recomputed states of one reverse-sweep segment in its own
// shared-memory slab, sized for the largest K in the batch.
#include "batch_mala.cuh"

namespace smc {

void count_launch();

__global__ void __launch_bounds__(kBatchMalaMaxThreads) k_mala_batch(const BatchMalaDev* __restrict__ mem,
                                                                     const BatchItem* __restrict__ items,
                                                                     int nitems, unsigned int* next,
                                                                     const int* iter)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ float Ls[kMaxD * kMaxD];
    __shared__ int s_it;
    __shared__ unsigned int acc_s;
    const int r = *iter;
    float* buf = reinterpret_cast<float*>(sm_raw) + threadIdx.x;
    for (;;) {
        if (threadIdx.x == 0) s_it = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int it = s_it;
        if (it >= nitems) break;   // the same value in every thread
        const BatchItem w = items[it];
        const BatchMalaDev& bm = mem[w.member];
        if (r >= bm.R) {
            __syncthreads();   // s_it is rewritten only after every thread has read it
            continue;
        }
        const int d = bm.a.m.d;
        for (int i = threadIdx.x; i < d * d; i += blockDim.x) Ls[i] = (float)bm.a.L[i];
        if (threadIdx.x == 0) acc_s = 0;
        __syncthreads();
        const int p = w.p0 + (int)threadIdx.x;
        bool acc = false;
        if (p < bm.a.P) {
            switch (bm.K * 8 + bm.I) {
#define SMC_MALA_BATCH_CASE(K, I)                                                                         \
    case K * 8 + I:                                                                                       \
        acc = mala_particle<GradEgarch<float, K, I>>(bm.a, (uint64_t)r, p, Ls, buf, (int)blockDim.x); \
        break;
                SMC_MALA_BATCH_CASE(1, 1) SMC_MALA_BATCH_CASE(1, 2) SMC_MALA_BATCH_CASE(1, 3) SMC_MALA_BATCH_CASE(1, 4)
                SMC_MALA_BATCH_CASE(2, 1) SMC_MALA_BATCH_CASE(2, 2) SMC_MALA_BATCH_CASE(2, 3) SMC_MALA_BATCH_CASE(2, 4)
                SMC_MALA_BATCH_CASE(3, 1) SMC_MALA_BATCH_CASE(3, 2) SMC_MALA_BATCH_CASE(3, 3) SMC_MALA_BATCH_CASE(3, 4)
                SMC_MALA_BATCH_CASE(4, 1) SMC_MALA_BATCH_CASE(4, 2) SMC_MALA_BATCH_CASE(4, 3) SMC_MALA_BATCH_CASE(4, 4)
#undef SMC_MALA_BATCH_CASE
            default: break;
            }
        }
        const unsigned int nacc = __popc(__ballot_sync(0xffffffffu, acc));
        if ((threadIdx.x & 31) == 0 && nacc) atomicAdd(&acc_s, nacc);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (acc_s) atomicAdd(bm.a.acc_count, (unsigned long long)acc_s);
            if (w.p0 == 0 && bm.a.pending) *bm.a.pending = 1;
        }
        __syncthreads();   // Ls, acc_s and s_it are reused by the next item
    }
}

size_t mala_batch_smem(int Kmax, int threads)
{
    return (size_t)GradEgarch<float, 1, 1>::kSeg * (size_t)(Kmax + 2) * (size_t)threads * sizeof(float);
}

cudaError_t mala_batch_occupancy(int threads, size_t smem, int* per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_mala_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_mala_batch, threads, smem);
}

cudaError_t launch_mala_batch(const BatchMalaDev* mem, const BatchItem* items, int nitems, unsigned int* next,
                              const int* iter, int grid, int threads, size_t smem, cudaStream_t s)
{
    k_mala_batch<<<grid, threads, smem, s>>>(mem, items, nitems, next, iter);
    count_launch();
    return cudaGetLastError();
}

}  // namespace smc
