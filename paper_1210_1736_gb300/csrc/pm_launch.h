// Launch interface between the C ABI (pm_api.cu) and the kernels, which are
// instantiated per precision in pm_fp32.cu and pm_fp64.cu.
#pragma once

#include <cuda_runtime.h>
#include "pm_internal.cuh"

#define PM_MAX_BATCH 16

// One FFT pass over every mass set of one geometry (gridDim.y = nsets).
struct FftArgs {
    const long long *rho[PM_MAX_BATCH];   // int64 densities (x forward pass)
    void *work[PM_MAX_BATCH];             // spectra, [z][y in 2ny][kx in nx+1]
    void *phi[PM_MAX_BATCH];              // potentials (x inverse pass)
    const void *hhat;                     // H-hat octant [nz+1][ny+1][nx+1]
    const void *tw;                       // exp(-2 pi i m / L), m < L
    int nx, ny, nz, P;                    // P = nx + 1
    long long nitems;                     // row pairs (x passes) or columns
    double scale;                         // 2^-s (x forward pass)
};

enum { COL_YFWD = 0, COL_ZCONV = 1, COL_YINV = 2 };

template <typename T> cudaError_t pm_set_attrs();
template <typename T> cudaError_t pm_launch_xfwd(const FftArgs &a, int nsets, cudaStream_t st);
template <typename T> cudaError_t pm_launch_col(const FftArgs &a, int mode, int nsets, cudaStream_t st);
template <typename T> cudaError_t pm_launch_xinv(const FftArgs &a, int nsets, cudaStream_t st);

template <typename T>
cudaError_t pm_launch_deposit(const PartK<T> &p, const SysK &sk, const CenK *cen, int aggregate, cudaStream_t st);
// mode: 0 kick-drift, 1 write accelerations, 2 kick only, 3 diagnostics
template <typename T>
cudaError_t pm_launch_force(int mode, const PartK<T> &p, const SysK &sk, const CenK *cen, double dt,
                            T *ax, T *ay, T *az, double *diag, cudaStream_t st);
// Recentring from the current positions (part: zeroed accumulators).
template <typename T>
cudaError_t pm_launch_recentre(const PartK<T> &p, const SysK &sk, CenK *cen, long long *part, cudaStream_t st);
template <typename T>
cudaError_t pm_launch_count_lost(const PartK<T> &p, unsigned long long *out, cudaStream_t st);
// Counting sort by spatial key; permutes p's arrays in place through scratch.
template <typename T>
cudaError_t pm_launch_sort(const PartK<T> &p, const PartK<T> &scratch, const SysK &sk, const CenK *cen,
                           const SortK &so, unsigned *count, unsigned *key, unsigned *rank, unsigned *bsum,
                           long long *perm, cudaStream_t st);

// FP64 H-hat construction (precision independent) and storage conversion.
cudaError_t pm_green_octant(double *h, int nx, int ny, int nz, double q, double h000, cudaStream_t st);
cudaError_t pm_axis_transform(const double *in, double *out, const double *cmat, int n1,
                              long long outer, long long inner, cudaStream_t st);
template <typename T>
cudaError_t pm_store_hhat(const double *in, T *out, long long n, double scale, cudaStream_t st);

// Records a message for pm_last_error() and returns code (C++ linkage; for
// translation units other than the C ABI file).
int pm_internal_fail(int code, const char *msg);
