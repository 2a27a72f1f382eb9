// CIC variant and adjoint kernels, both precisions.
#include "pm_launch.h"
#include "pm_cic.cuh"
PM_CIC_INSTANTIATE(float)
PM_CIC_INSTANTIATE(double)
