// Disc diagnostics kernels, both precisions.
#include "pm_diag.cuh"
PM_DIAG_INSTANTIATE(float)
PM_DIAG_INSTANTIATE(double)
