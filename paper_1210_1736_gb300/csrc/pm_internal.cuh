// Internal types and device helpers of the particle-mesh library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pm.h"

#define PM_SETS 5

template <typename T> struct cplx_t;
template <> struct cplx_t<float>  { typedef float2  type; };
template <> struct cplx_t<double> { typedef double2 type; };

// Geometry as the particle kernels see it.  gxy/gz are (float)(1/l): the
// canonical FP32 cell-assignment factors; the rest are FP64 lengths and
// finite-difference coefficients of Eq. (eqn:diff).
struct GeomK {
    int nx, ny, nz;
    float gxy, gz;
    double lxy, lz;
    double c_gx, c_gz;     // 1/(2 l_xy), 1/(2 l_z)         central difference
    double c_hxx, c_hzz;   // 1/l_xy^2, 1/l_z^2              second difference
    double c_mxy, c_mxz;   // 1/(4 l_xy l_xy), 1/(4 l_xy l_z) mixed difference
    // the same rounded to FP32, so that FP32 kernels convert nothing per
    // particle (double arithmetic, conversions included, is slow on GB300)
    float flxy, flz, fc_gx, fc_gz, fc_hxx, fc_hzz, fc_mxy, fc_mxz;
    float fil_xy, fil_z;   // (float)(1/l_xy), (float)(1/l_z)
};

// A geometry coefficient in the working precision: the FP64 value for
// double kernels, its FP32 copy for float kernels.
template <typename T> __device__ __forceinline__ T pick(double d, float f);
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }

struct GalK {
    GeomK fine, med, coarse;   // nx == 0: absent
    float rc2, ro2;            // (float)(r_core^2), (float)(r_out^2)
    int recentre, sD;          // recentring flag, offset fixed-point shift
    unsigned long long *rho[PM_SETS];   // int64 densities (two's complement)
    // potentials in the context precision, combined as the force stencils
    // read them (combination rule of Sec. 2.1)
    const void *phi_fine;   // Phi_1
    const void *phi_m3;     // Phi_3
    const void *phi_m23;    // Phi_2 + Phi_3
    const void *phi_c5;     // Phi_5
    const void *phi_call;   // Phi_4 + Phi_5 (Phi_5 when there is no medium grid)
    // forward differences of Phi_1 (fx[i] = Phi_1[i+1] - Phi_1[i], likewise
    // fy, fz), from which the fine-grid force is built (null: use Phi_1)
    const void *fd_x, *fd_y, *fd_z;
};

struct SysK {
    int ngal;
    float rsys2;
    double sc[3];
    float sc_hi[3], sc_lo[3];  // system centre split as fl32(c) + fl32(c - fl32(c))
    double mscale;             // 2^s
    float mscale_f;            // 2^s as float (exact)
    GalK gal[PM_MAX_GALAXIES];
};

// Centres of grids 1-3: FP64 values and their FP32 split (hi, lo) per axis.
struct CenK {
    double c[PM_MAX_GALAXIES][3];
    float hi[PM_MAX_GALAXIES][3];
    float lo[PM_MAX_GALAXIES][3];
};

// Key layout of the spatial sort: per galaxy and region (core, shell, outer)
// a base offset and the bin shift applied to the cell indices of that
// region's grid (fine, medium, coarse); the last key collects lost particles.
struct SortK {
    long long base[PM_MAX_GALAXIES][3];
    int shift[PM_MAX_GALAXIES][3];
    long long nkeys;
};

template <typename T> struct PartK {
    T *x, *y, *z, *vx, *vy, *vz;
    const T *m;
    const int32_t *gal;
    uint32_t *flags;
    long long n;
};

// ----------------------------------------------------------------------------
// Canonical cell assignment (Eq. eqn:cell).  Every rounding is explicit and
// no multiply-add is fused, so these functions and the CPU reference agree
// bit for bit: the offset d from a centre c (pm_canon), then
// u = fl32(fl32(d*gamma) + N/2), a = floor(fl32(u + 1/2)).
// ----------------------------------------------------------------------------
__device__ __forceinline__ float pm_off32(double x, double c) {
    return __double2float_rn(__dsub_rn(x, c));
}
// FP32 contexts: positions are floats and the offset is
// fl32(fl32(x - c_hi) - c_lo) with c = c_hi + c_lo, no FP64 arithmetic.
__device__ __forceinline__ float pm_off32s(float x, float chi, float clo) {
    return __fsub_rn(__fsub_rn(x, chi), clo);
}
// Canonical offset for the context precision.
__device__ __forceinline__ float pm_canon(float x, double, float chi, float clo) { return pm_off32s(x, chi, clo); }
__device__ __forceinline__ float pm_canon(double x, double c, float, float) { return pm_off32(x, c); }
// Fixed-point mass q = rint(m 2^s): for float m the product is exact in FP32.
__device__ __forceinline__ long long pm_qmass(float m, double, float sf) { return __float2ll_rn(__fmul_rn(m, sf)); }
__device__ __forceinline__ long long pm_qmass(double m, double s, float) { return __double2ll_rn(__dmul_rn(m, s)); }
__device__ __forceinline__ int pm_cell(float d, float g, int n) {
    float u = __fadd_rn(__fmul_rn(d, g), (float)(n >> 1));
    return (int)floorf(__fadd_rn(u, 0.5f));
}
__device__ __forceinline__ float pm_r2(float dx, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}
__device__ __forceinline__ bool pm_inbox(int a, int n) { return a >= 2 && a <= n - 3; }

struct Cell { int i, j, k; bool ok; };

__device__ __forceinline__ Cell pm_cells(const GeomK &g, float dx, float dy, float dz) {
    Cell c;
    c.i = pm_cell(dx, g.gxy, g.nx);
    c.j = pm_cell(dy, g.gxy, g.ny);
    c.k = pm_cell(dz, g.gz, g.nz);
    c.ok = pm_inbox(c.i, g.nx) && pm_inbox(c.j, g.ny) && pm_inbox(c.k, g.nz);
    return c;
}

enum { REG_CORE = 0, REG_SHELL = 1, REG_OUTER = 2 };

// Region of a point relative to galaxy G centred on c (Sec. 2.1): core =
// r < R_core inside grids 1 and 2; shell = not core, r < R_out inside grid 2.
// Returns the fine and medium cells as a by-product.
__device__ __forceinline__ int pm_region(const GalK &G, float dx, float dy, float dz,
                                         Cell &cf, Cell &cm) {
    float r2 = pm_r2(dx, dy, dz);
    cm.ok = false; cf.ok = false;
    // at or beyond R_out neither test below can pass (rc2 <= ro2, as
    // R_core <= R_out and rounding to FP32 is monotonic): outer, whatever
    // the cells (a NaN distance lands here as it did through them)
    if (!(r2 < G.ro2)) return REG_OUTER;
    if (G.med.nx) cm = pm_cells(G.med, dx, dy, dz);
    if (G.fine.nx && G.med.nx) {
        cf = pm_cells(G.fine, dx, dy, dz);
        if (r2 < G.rc2 && cf.ok && cm.ok) return REG_CORE;
    }
    if (G.med.nx && r2 < G.ro2 && cm.ok) return REG_SHELL;
    return REG_OUTER;
}

// ----------------------------------------------------------------------------
// Small complex helpers
// ----------------------------------------------------------------------------
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// FP32: one packed two-lane instruction (sm_100 family) per complex add or
// subtract, rounded per component as the scalar operations (bit-identical);
// the FFT passes are bound by instruction issue.
template <> __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cconjmul(C a, C b) {  // a * conj(b)
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }
// multiply by SIGN*i
template <int SIGN, typename C> __device__ __forceinline__ C cmul_i(C z) {
    C r;
    if (SIGN > 0) { r.x = -z.y; r.y = z.x; } else { r.x = z.y; r.y = -z.x; }
    return r;
}
