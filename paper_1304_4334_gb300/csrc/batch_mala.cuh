// Batched driver pieces shared by the random-walk and MALA persistent kernels
// (batch.cu, batch_mala.cu).  Not part of the C ABI.
#pragma once

#include "mala.cuh"

namespace smc {

// A work item of the persistent M-phase kernels: one tile of a dataset's particles.
struct BatchItem {
    int member, p0;
};

// Per-dataset MALA arguments of the current cycle and its iteration count R.
struct BatchMalaDev {
    MalaArgs a;
    int K, I, R;
};

// Threads per block of the batched MALA kernel (each thread holds a
// reverse-sweep segment slab in shared memory, as the single-run kernel does).
constexpr int kBatchMalaMaxThreads = 64;

// Dynamic shared memory of a block of `threads` threads for models up to Kmax.
size_t mala_batch_smem(int Kmax, int threads);
// Resident blocks per SM (also raises the kernel's dynamic shared-memory limit).
cudaError_t mala_batch_occupancy(int threads, size_t smem, int* per_sm);
cudaError_t launch_mala_batch(const BatchMalaDev* mem, const BatchItem* items, int nitems, unsigned int* next,
                              const int* iter, int grid, int threads, size_t smem, cudaStream_t s);

}  // namespace smc
