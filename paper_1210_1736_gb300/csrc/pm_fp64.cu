// FP64 instantiation of the kernels (the plain FP64 path).
#include "pm_kernels.cuh"
PM_INSTANTIATE(double)
