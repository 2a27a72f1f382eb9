// Per-particle helpers shared by the particle kernels of the NGP step and of
// its CIC variant.
#pragma once

#include "pm_internal.cuh"

namespace pmk {

__device__ __forceinline__ size_t cell_off(const GeomK &g, const Cell &c) {
    return ((size_t)c.k * g.ny + c.j) * g.nx + c.i;
}

struct Cen1 {
    double c[3];
    float hi[3], lo[3];
};
__device__ __forceinline__ Cen1 load_cen(const CenK *cen, int g) {
    Cen1 r;
    const CenK *cs = cen;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r.c[k] = __ldg(&cs->c[g][k]);
        r.hi[k] = __ldg(&cs->hi[g][k]);
        r.lo[k] = __ldg(&cs->lo[g][k]);
    }
    return r;
}

// Offset used for Delta in Eq. (eqn:diff): the canonical FP32 offset in FP32
// contexts, the exact FP64 difference in FP64 contexts.
__device__ __forceinline__ float rel_off(float x, double, float chi, float clo) { return pm_off32s(x, chi, clo); }
__device__ __forceinline__ double rel_off(double x, double c, float, float) { return __dsub_rn(x, c); }

// Offset of a particle from the centre of its cell (Delta of Eq. eqn:diff).
template <typename T>
__device__ __forceinline__ void cell_delta(const GeomK &g, const Cell &cl, T rx, T ry, T rz, T &dx, T &dy, T &dz) {
    dx = rx - (T)(cl.i - (g.nx >> 1)) * pick<T>(g.lxy, g.flxy);
    dy = ry - (T)(cl.j - (g.ny >> 1)) * pick<T>(g.lxy, g.flxy);
    dz = rz - (T)(cl.k - (g.nz >> 1)) * pick<T>(g.lz, g.flz);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}


}  // namespace pmk
