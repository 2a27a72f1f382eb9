// FP32 instantiation of the kernels (the batched production path).
#include "pm_kernels.cuh"
PM_INSTANTIATE(float)
