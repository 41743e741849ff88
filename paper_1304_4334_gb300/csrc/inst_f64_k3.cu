// FP64 EGARCH kernels with K = 3 volatility factors, I = 1..4 mixture components.
#include "inst_egarch.cuh"
SMC_INSTANTIATE_EGARCH(f64, PolicyEgarchF64, PolicyEgarchF64, 3)
