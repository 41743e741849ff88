// FP32 EGARCH kernels with K = 1 volatility factors, I = 1..4 mixture components.
#include "inst_egarch.cuh"
SMC_INSTANTIATE_EGARCH(f32, PolicyEgarchF32, 1)
