// Disc diagnostics of the paper's Sec. 6 (thickness sqrt<z^2>(R), heat
// E_heat about the binned circular velocity, velocity dispersions in an
// annulus, Fourier modes A~_m in rings) as FP64 reductions over the selected
// particles, positions and velocities taken relative to a galaxy centre.
//
// Radial bins of equal particle numbers are bounded by exact order
// statistics of R^2: an MSD radix select over the IEEE bits of R^2 (a
// non-negative double, so its bits order like its value), 8 bits per pass,
// one histogram per distinct prefix of the boundaries still being resolved.
#pragma once

#include "pm_launch.h"
#include "pm_particle.cuh"

namespace pmk {

template <typename T>
__device__ __forceinline__ bool diag_take(const DiagP<T> &d, long long i) {
    if (d.flags[i] & PM_FLAG_LOST) return false;
    return d.sel ? d.sel[i] != 0 : d.gal_id[i] == d.gal;
}

// R^2 with the same operations as the FP64 reference (no contraction).
template <typename T>
__device__ __forceinline__ double diag_r2(const DiagP<T> &d, long long i, double &dx, double &dy) {
    dx = __dsub_rn((double)d.x[i], d.c[0]);
    dy = __dsub_rn((double)d.y[i], d.c[1]);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// One pass of the radix select: particles whose key agrees with one of the
// npref sorted prefixes (the key's top 8*pass bits) count their next digit.
template <typename T>
__global__ void __launch_bounds__(256) k_diag_hist(DiagP<T> d, int pass, const unsigned long long *pref, int npref,
                                                   unsigned *hist) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += stride) {
        if (!diag_take(d, i)) continue;
        double dx, dy;
        const unsigned long long key = (unsigned long long)__double_as_longlong(diag_r2(d, i, dx, dy));
        int j = 0;
        if (pass > 0) {
            const unsigned long long pk = key >> (64 - 8 * pass);
            int lo = 0, hi = npref - 1;
            j = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                if (pref[mid] == pk) { j = mid; break; }
                if (pref[mid] < pk) lo = mid + 1; else hi = mid - 1;
            }
            if (j < 0) continue;
        }
        atomicAdd(hist + j * 256 + (int)((key >> (56 - 8 * pass)) & 255u), 1u);
    }
}

__device__ __forceinline__ void diag_add(double *sh, int k, double v) { atomicAdd(sh + k, v); }

template <typename T>
__global__ void __launch_bounds__(256) k_diag_sums(DiagP<T> d, DiagQ q, const unsigned long long *edges,
                                                   double *acc) {
    extern __shared__ double sh[];
    const int nacc = 4 * q.nbins + 7 + 2 * q.nring * q.mmax;
    for (int k = threadIdx.x; k < nacc; k += blockDim.x) sh[k] = 0.0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += stride) {
        if (!diag_take(d, i)) continue;
        double dx, dy;
        const double r2 = diag_r2(d, i, dx, dy);
        const unsigned long long key = (unsigned long long)__double_as_longlong(r2);
        int b = 0;   // number of edges <= key
        {
            int lo = 0, hi = q.nbins - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (edges[mid] <= key) lo = mid + 1; else hi = mid;
            }
            b = lo;
        }
        const double R = __dsqrt_rn(r2);
        const double dz = __dsub_rn((double)d.z[i], d.c[2]);
        const double vx = d.vx[i], vy = d.vy[i], vz = d.vz[i], m = d.m[i];
        const double vR = R > 0 ? (dx * vx + dy * vy) / R : 0.0;
        const double vphi = R > 0 ? (dx * vy - dy * vx) / R : 0.0;
        diag_add(sh, 4 * b + 0, R);
        diag_add(sh, 4 * b + 1, 1.0);
        diag_add(sh, 4 * b + 2, dz * dz);
        diag_add(sh, 4 * b + 3, vphi);
        if (R >= q.rlo && R < q.rhi) {
            double *a = sh + 4 * q.nbins;
            diag_add(a, 0, m);
            diag_add(a, 1, m * vR);
            diag_add(a, 2, m * vR * vR);
            diag_add(a, 3, m * vphi);
            diag_add(a, 4, m * vphi * vphi);
            diag_add(a, 5, m * vz);
            diag_add(a, 6, m * vz * vz);
        }
        if (R > 0 && R < q.r_ring) {
            const int ring = (int)floor(__ddiv_rn(R, q.width));
            if (ring < q.nring) {
                double *a = sh + 4 * q.nbins + 7 + 2 * ring * q.mmax;
                // exp(-i m phi) by the angle-addition recurrence from cos, sin phi
                const double c1 = dx / R, s1 = dy / R;
                double cm = c1, sm = s1;
                for (int mo = 0; mo < q.mmax; ++mo) {
                    diag_add(a, 2 * mo, m * cm);
                    diag_add(a, 2 * mo + 1, -m * sm);
                    const double cn = cm * c1 - sm * s1;
                    sm = sm * c1 + cm * s1;
                    cm = cn;
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nacc; k += blockDim.x)
        if (sh[k] != 0.0) atomicAdd(acc + k, sh[k]);
}

// E_heat with vbar_c linear in R between (xp[k], fp[k]), k < np, held
// constant outside.
template <typename T>
__global__ void __launch_bounds__(256) k_diag_heat(DiagP<T> d, const double *xp, const double *fp, int np,
                                                   double *acc) {
    double e = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += stride) {
        if (!diag_take(d, i)) continue;
        double dx, dy;
        const double R = __dsqrt_rn(diag_r2(d, i, dx, dy));
        const double vx = d.vx[i], vy = d.vy[i], vz = d.vz[i];
        const double vR = R > 0 ? (dx * vx + dy * vy) / R : 0.0;
        const double vphi = R > 0 ? (dx * vy - dy * vx) / R : 0.0;
        double vb;
        if (R <= xp[0]) vb = fp[0];
        else if (R >= xp[np - 1]) vb = fp[np - 1];
        else {
            int lo = 0, hi = np - 1;   // xp[lo] < R < xp[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (xp[mid] <= R) lo = mid; else hi = mid;
            }
            vb = (fp[hi] - fp[lo]) / (xp[hi] - xp[lo]) * (R - xp[lo]) + fp[lo];
        }
        const double dv = vphi - vb;
        e += 0.5 * (double)d.m[i] * (vR * vR + dv * dv + vz * vz);
    }
    __shared__ double red[8];
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(acc, s);
    }
}

}  // namespace pmk

template <typename T> cudaError_t pm_launch_diag_hist(const pmk::DiagP<T> &d, int pass, const unsigned long long *pref,
                                                      int npref, unsigned *hist, cudaStream_t st) {
    if (d.n <= 0) return cudaSuccess;
    long long b = (d.n + 255) / 256;
    pmk::k_diag_hist<T><<<(int)(b < 4096 ? b : 4096), 256, 0, st>>>(d, pass, pref, npref, hist);
    return cudaGetLastError();
}
template <typename T> cudaError_t pm_launch_diag_sums(const pmk::DiagP<T> &d, const pmk::DiagQ &q,
                                                      const unsigned long long *edges, double *acc,
                                                      cudaStream_t st) {
    if (d.n <= 0) return cudaSuccess;
    const size_t sh = sizeof(double) * (4 * q.nbins + 7 + 2 * q.nring * q.mmax);
    long long b = (d.n + 255) / 256;
    pmk::k_diag_sums<T><<<(int)(b < 1024 ? b : 1024), 256, sh, st>>>(d, q, edges, acc);
    return cudaGetLastError();
}
template <typename T> cudaError_t pm_launch_diag_heat(const pmk::DiagP<T> &d, const double *xp, const double *fp,
                                                      int np, double *acc, cudaStream_t st) {
    if (d.n <= 0) return cudaSuccess;
    long long b = (d.n + 255) / 256;
    pmk::k_diag_heat<T><<<(int)(b < 1024 ? b : 1024), 256, 0, st>>>(d, xp, fp, np, acc);
    return cudaGetLastError();
}

#define PM_DIAG_INSTANTIATE(T)                                                                                 \
    template cudaError_t pm_launch_diag_hist<T>(const pmk::DiagP<T> &, int, const unsigned long long *, int,   \
                                                unsigned *, cudaStream_t);                                     \
    template cudaError_t pm_launch_diag_sums<T>(const pmk::DiagP<T> &, const pmk::DiagQ &,                     \
                                                const unsigned long long *, double *, cudaStream_t);          \
    template cudaError_t pm_launch_diag_heat<T>(const pmk::DiagP<T> &, const double *, const double *, int,    \
                                                double *, cudaStream_t);
