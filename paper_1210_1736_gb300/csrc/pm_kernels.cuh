// Kernels of the nested-grid particle-mesh step, templated on the working
// precision T (float or double).  Included once per precision.
#pragma once

#include <utility>

#include "pm_passes.cuh"
#include "pm_particle.cuh"

namespace pmk {

// ---------------------------------------------------------------------------
// Particle kernels.  The system description is a __grid_constant__ kernel
// parameter (read through the constant cache, no staging); the centres of
// grids 1-3 are read from device memory.
// ---------------------------------------------------------------------------
// Adds q (two's complement int64) to *addr for every lane with active set.
// After the spatial sort, lanes that target the same cell are mostly
// adjacent: the runs of adjacent active lanes with one address are found
// with one shuffle of the address and a ballot, each run is summed by a
// segmented inclusive scan over shuffles (64-bit adds, exact mod 2^64; it
// stops as soon as no run in the warp is longer than the distance reached),
// and the run's last lane issues one atomic.  Lanes with one address that
// are not adjacent form separate runs (still exact).  Every lane of the warp
// must call it.
__device__ __forceinline__ void agg_add(unsigned long long *addr, unsigned long long q, bool active) {
    const unsigned FULL = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31);
    const unsigned long long key = active ? (unsigned long long)addr : 0ull;   // no cell lives at address 0
    const unsigned long long prev = __shfl_up_sync(FULL, key, 1);
    const bool head = active && (lane == 0 || prev != key);
    // run boundaries: run heads and inactive lanes (an active lane after an
    // inactive one is a head, since its key is not 0)
    const unsigned brk = __ballot_sync(FULL, head) | ~__ballot_sync(FULL, active);
    const unsigned upto = lane == 31 ? FULL : ((2u << lane) - 1u);   // lanes 0..lane
    const int h = 31 - __clz(brk & upto);                            // this run's head
    unsigned long long v = active ? q : 0ull;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const bool take = lane - d >= h;
        if (!__any_sync(FULL, take)) break;
        const unsigned long long u = __shfl_up_sync(FULL, v, d);
        if (take) v += u;
    }
    if (active && (lane == 31 || ((brk >> (lane + 1)) & 1u))) atomicAdd(addr, v);
}

// Steps a2-a3: classification and exact fixed-point mass assignment.  The
// loop is warp-uniform so the aggregation can use warp collectives.
template <typename T>
__global__ void __launch_bounds__(256, 6) k_deposit(PartK<T> p, const __grid_constant__ SysK s, const CenK *cen,
                                                 int aggregate) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < p.n; b += stride) {
        const long long i = b + threadIdx.x;
        unsigned long long *tgt[3] = {nullptr, nullptr, nullptr};
        unsigned long long q = 0;
        if (i < p.n) {
            // all loads of the particle before the flag test
            const uint32_t f = p.flags[i];
            const T x = p.x[i], y = p.y[i], z = p.z[i], mi = p.m[i];
            const int g = p.gal[i];
            if (!(f & PM_FLAG_LOST)) {
                const float sx = pm_canon(x, s.sc[0], s.sc_hi[0], s.sc_lo[0]);
                const float sy = pm_canon(y, s.sc[1], s.sc_hi[1], s.sc_lo[1]);
                const float sz = pm_canon(z, s.sc[2], s.sc_hi[2], s.sc_lo[2]);
                bool lost = !(pm_r2(sx, sy, sz) < s.rsys2);
                if (g < 0 || g >= s.ngal) lost = true;
                Cell cc;
                cc.i = cc.j = cc.k = 0; cc.ok = false;
                for (int h = 0; h < s.ngal; ++h) {
                    const Cell ch = pm_cells(s.gal[h].coarse, sx, sy, sz);
                    lost = lost || !ch.ok;
                    if (h == g) cc = ch;
                }
                if (lost) {
                    p.flags[i] = f | PM_FLAG_LOST;
                } else {
                    const GalK &G = s.gal[g];
                    const Cen1 ce = load_cen(cen, g);
                    const float dx = pm_canon(x, ce.c[0], ce.hi[0], ce.lo[0]);
                    const float dy = pm_canon(y, ce.c[1], ce.hi[1], ce.lo[1]);
                    const float dz = pm_canon(z, ce.c[2], ce.hi[2], ce.lo[2]);
                    Cell cf, cm;
                    const int reg = pm_region(G, dx, dy, dz, cf, cm);
                    q = (unsigned long long)pm_qmass(mi, s.mscale, s.mscale_f);
                    if (reg == REG_CORE) {
                        tgt[0] = G.rho[0] + cell_off(G.fine, cf);
                        tgt[1] = G.rho[1] + cell_off(G.med, cm);
                        tgt[2] = G.rho[3] + cell_off(G.coarse, cc);
                    } else if (reg == REG_SHELL) {
                        tgt[1] = G.rho[2] + cell_off(G.med, cm);
                        tgt[2] = G.rho[3] + cell_off(G.coarse, cc);
                    } else {
                        tgt[2] = G.rho[4] + cell_off(G.coarse, cc);
                    }
                }
            }
        }
        if (aggregate) {
#pragma unroll
            for (int t = 0; t < 3; ++t) agg_add(tgt[t], q, tgt[t] != nullptr);
        } else {
#pragma unroll
            for (int t = 0; t < 3; ++t)
                if (tgt[t]) atomicAdd(tgt[t], q);
        }
    }
}

// Eq. (eqn:diff) on one grid (with an optional second potential on the same
// grid summed point by point), accumulated into acc; optionally the
// potential at the particle (cell value + gradient . Delta).
template <typename T>
__device__ __forceinline__ void stencil(const GeomK &g, const T *__restrict__ P1, const T *__restrict__ P2,
                                        const Cell &cl, T dx, T dy, T dz, T *acc, T *phi) {
    const int sy = g.nx, sz = g.nx * g.ny;   // a grid has at most 256^3 cells: 32-bit offsets
    const size_t base = cell_off(g, cl);
    const T *b1 = P1 + base;
    const T *b2 = P2 ? P2 + base : nullptr;
    auto ld = [&](int di, int dj, int dk) -> T {
        const int o = di + dj * sy + dk * sz;
        T v = __ldg(b1 + o);
        if (b2) v += __ldg(b2 + o);
        return v;
    };
    const T p0 = ld(0, 0, 0);
    const T xp = ld(1, 0, 0), xm = ld(-1, 0, 0);
    const T yp = ld(0, 1, 0), ym = ld(0, -1, 0);
    const T zp = ld(0, 0, 1), zm = ld(0, 0, -1);
    const T mxy = (ld(1, 1, 0) - ld(-1, 1, 0) + ld(-1, -1, 0) - ld(1, -1, 0)) * pick<T>(g.c_mxy, g.fc_mxy);
    const T mxz = (ld(1, 0, 1) - ld(-1, 0, 1) + ld(-1, 0, -1) - ld(1, 0, -1)) * pick<T>(g.c_mxz, g.fc_mxz);
    const T myz = (ld(0, 1, 1) - ld(0, -1, 1) + ld(0, -1, -1) - ld(0, 1, -1)) * pick<T>(g.c_mxz, g.fc_mxz);
    const T gx = (xp - xm) * pick<T>(g.c_gx, g.fc_gx), gy = (yp - ym) * pick<T>(g.c_gx, g.fc_gx), gz = (zp - zm) * pick<T>(g.c_gz, g.fc_gz);
    const T hxx = (xp + xm - 2 * p0) * pick<T>(g.c_hxx, g.fc_hxx);
    const T hyy = (yp + ym - 2 * p0) * pick<T>(g.c_hxx, g.fc_hxx);
    const T hzz = (zp + zm - 2 * p0) * pick<T>(g.c_hzz, g.fc_hzz);
    acc[0] += gx + hxx * dx + mxy * dy + mxz * dz;
    acc[1] += gy + hyy * dy + mxy * dx + myz * dz;
    acc[2] += gz + hzz * dz + mxz * dx + myz * dy;
    if (phi) *phi += p0 + gx * dx + gy * dy + gz * dz;
}

// Eq. (eqn:diff) on grid 1 from the forward differences of Phi_1,
// fx[i] = Phi[i+1] - Phi[i] (and fy, fz), which the convolution returns
// directly; their FP32 rounding is relative to the differences, not to Phi.
// With f(di, dj, dk) = f at the cell (i+di, j+dj, k+dk):
//   Phi(1) - Phi(-1)          = fx(0) + fx(-1)
//   Phi(1) + Phi(-1) - 2Phi(0) = fx(0) - fx(-1)
//   Phi(1,1) - Phi(-1,1) + Phi(-1,-1) - Phi(1,-1)
//                             = fx(0,1) + fx(-1,1) - fx(0,-1) - fx(-1,-1)
// and likewise for the other mixed terms and components (each component's
// terms from its own difference field).
template <typename T>
__device__ __forceinline__ void stencil_diff(const GeomK &g, const T *__restrict__ FX, const T *__restrict__ FY,
                                             const T *__restrict__ FZ, const Cell &cl, T dx, T dy, T dz, T *acc) {
    const int sy = g.nx, sz = g.nx * g.ny;
    const size_t base = cell_off(g, cl);
    const T *bx = FX + base, *by = FY + base, *bz = FZ + base;
    auto o = [&](int di, int dj, int dk) { return di + dj * sy + dk * sz; };
    const T cg = pick<T>(g.c_gx, g.fc_gx), cgz = pick<T>(g.c_gz, g.fc_gz);
    const T chx = pick<T>(g.c_hxx, g.fc_hxx), chz = pick<T>(g.c_hzz, g.fc_hzz);
    const T cmxy = pick<T>(g.c_mxy, g.fc_mxy), cmxz = pick<T>(g.c_mxz, g.fc_mxz);
    const T x0 = __ldg(bx), xm = __ldg(bx + o(-1, 0, 0));
    const T xyp = __ldg(bx + o(0, 1, 0)) + __ldg(bx + o(-1, 1, 0));
    const T xym = __ldg(bx + o(0, -1, 0)) + __ldg(bx + o(-1, -1, 0));
    const T xzp = __ldg(bx + o(0, 0, 1)) + __ldg(bx + o(-1, 0, 1));
    const T xzm = __ldg(bx + o(0, 0, -1)) + __ldg(bx + o(-1, 0, -1));
    const T y0 = __ldg(by), ym = __ldg(by + o(0, -1, 0));
    const T yxp = __ldg(by + o(1, 0, 0)) + __ldg(by + o(1, -1, 0));
    const T yxm = __ldg(by + o(-1, 0, 0)) + __ldg(by + o(-1, -1, 0));
    const T yzp = __ldg(by + o(0, 0, 1)) + __ldg(by + o(0, -1, 1));
    const T yzm = __ldg(by + o(0, 0, -1)) + __ldg(by + o(0, -1, -1));
    const T z0 = __ldg(bz), zm = __ldg(bz + o(0, 0, -1));
    const T zxp = __ldg(bz + o(1, 0, 0)) + __ldg(bz + o(1, 0, -1));
    const T zxm = __ldg(bz + o(-1, 0, 0)) + __ldg(bz + o(-1, 0, -1));
    const T zyp = __ldg(bz + o(0, 1, 0)) + __ldg(bz + o(0, 1, -1));
    const T zym = __ldg(bz + o(0, -1, 0)) + __ldg(bz + o(0, -1, -1));
    acc[0] += (x0 + xm) * cg + (x0 - xm) * chx * dx + (xyp - xym) * cmxy * dy + (xzp - xzm) * cmxz * dz;
    acc[1] += (y0 + ym) * cg + (y0 - ym) * chx * dy + (yxp - yxm) * cmxy * dx + (yzp - yzm) * cmxz * dz;
    acc[2] += (z0 + zm) * cgz + (z0 - zm) * chz * dz + (zxp - zxm) * cmxz * dx + (zyp - zym) * cmxz * dy;
}

// ---------------------------------------------------------------------------
// Step a1 (recentring).  The centre of mass of each recentring galaxy's live
// particles within R_core of its centre c is accumulated exactly in integers:
// sum M and sum M*D with M = q >> 26 and D = rint(d 2^sD) (|D| < 2^24); then
// c' = c + (sum M D / sum M) 2^-sD.  Warp sums go to shared memory, each
// block adds its sums into one of COM_SLOTS accumulator rows, and a one-block
// kernel adds the rows and moves the centres.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int com_contrib(const SysK &s, const CenK *cen, int g, T x, T y, T z, T m,
                                           long long &M, int &Dx, int &Dy, int &Dz) {
    if (g < 0 || g >= s.ngal || !s.gal[g].recentre) return -1;
    const Cen1 ce = load_cen(cen, g);
    const float dx = pm_canon(x, ce.c[0], ce.hi[0], ce.lo[0]);
    const float dy = pm_canon(y, ce.c[1], ce.hi[1], ce.lo[1]);
    const float dz = pm_canon(z, ce.c[2], ce.hi[2], ce.lo[2]);
    if (!(pm_r2(dx, dy, dz) < s.gal[g].rc2)) return -1;
    M = pm_qmass(m, s.mscale, s.mscale_f) >> 26;
    const float sc = __int_as_float((127 + s.gal[g].sD) << 23);  // 2^sD
    Dx = __float2int_rn(__fmul_rn(dx, sc));
    Dy = __float2int_rn(__fmul_rn(dy, sc));
    Dz = __float2int_rn(__fmul_rn(dz, sc));
    return g;
}

// Read-only global loads the compiler keeps where they are written.
__device__ __forceinline__ float ld_early(const float *q) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ double ld_early(const double *q) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ int ld_early(const int32_t *q) {
    int v;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ uint32_t ld_early(const uint32_t *q) {
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(q));
    return v;
}

// Exact warp sum of a two's complement int64 (mod 2^64) from three chunk
// reductions of 22, 21 and 21 bits (each chunk sum stays below 2^32).
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    const unsigned FULL = 0xffffffffu;
    const unsigned s0 = __reduce_add_sync(FULL, (unsigned)(v & 0x3fffffu));
    const unsigned s1 = __reduce_add_sync(FULL, (unsigned)((v >> 22) & 0x1fffffu));
    const unsigned s2 = __reduce_add_sync(FULL, (unsigned)(v >> 43));
    return (unsigned long long)s0 + ((unsigned long long)s1 << 22) + ((unsigned long long)s2 << 43);
}

// Warp-collective: every lane of the warp calls it with its sums (M, M Dx,
// M Dy, M Dz, mod 2^64) for galaxy g (g = -1: no contribution).
__device__ __forceinline__ void com_warp_add(const SysK &s, unsigned long long (*red)[4], int g,
                                             const unsigned long long (&S)[4]) {
    for (int h = 0; h < s.ngal; ++h) {
        if (!__any_sync(0xffffffffu, g == h)) continue;
        const bool mine = (g == h);
        unsigned long long v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = warp_sum_u64(mine ? S[k] : 0ull);
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&red[h][k], v[k]);
    }
}

// Block epilogue: the block's sums are added (integer atomics, any order)
// into one of COM_SLOTS accumulator rows, part[blockIdx % COM_SLOTS][galaxy][4],
// so no address sees more than a few dozen atomics.
constexpr int COM_SLOTS = 64;
__device__ __forceinline__ void com_write_partials(const SysK &s, unsigned long long (*red)[4], long long *part) {
    __syncthreads();
    if (threadIdx.x < s.ngal * 4) {
        const unsigned long long v = (&red[0][0])[threadIdx.x];
        if (v) atomicAdd(reinterpret_cast<unsigned long long *>(part) + (blockIdx.x % COM_SLOTS) * PM_MAX_GALAXIES * 4 +
                             threadIdx.x, v);
    }
}

// One thread's running sums for galaxy g straight into its block's row.
__device__ __forceinline__ void com_flush(long long *part, int g, unsigned long long (&S)[4]) {
    unsigned long long *row = reinterpret_cast<unsigned long long *>(part) +
                              (blockIdx.x % COM_SLOTS) * PM_MAX_GALAXIES * 4 + g * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (S[k]) atomicAdd(row + k, S[k]);
        S[k] = 0;
    }
}

// One block of 256 threads: adds the COM_SLOTS accumulator rows, clears them
// for the next use, and moves the centres: c += (sum M D / sum M) 2^-sD.
static __global__ void __launch_bounds__(256) k_com_apply(const __grid_constant__ SysK s, long long *part,
                                                          CenK *cen) {
    constexpr int NV = COM_SLOTS * PM_MAX_GALAXIES * 4;  // 2048 values, value index = slot * 32 + v
    __shared__ long long red2[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long acc = 0;
#pragma unroll
    for (int k = 0; k < NV / 256; ++k) {
        long long *q = part + threadIdx.x + 256 * k;   // v = threadIdx.x % 32 for every k
        acc += *q;
        *q = 0;
    }
    red2[w][lane] = acc;
    __syncthreads();
    const int g = threadIdx.x;
    if (g >= s.ngal || !s.gal[g].recentre) return;
    long long S[4];
    for (int k = 0; k < 4; ++k) {
        S[k] = 0;
        for (int q = 0; q < 8; ++q) S[k] += red2[q][4 * g + k];
    }
    if (S[0] <= 0) return;
    const double sc = ldexp(1.0, -s.gal[g].sD);
    for (int k = 0; k < 3; ++k) {
        const double c =
            __dadd_rn(cen->c[g][k], __dmul_rn(__ddiv_rn(__ll2double_rn(S[1 + k]), __ll2double_rn(S[0])), sc));
        const float hi = __double2float_rn(c);
        cen->c[g][k] = c;
        cen->hi[g][k] = hi;
        cen->lo[g][k] = __double2float_rn(__dsub_rn(c, (double)hi));
    }
}

// Step a1: centre-of-mass sums of the current positions, then k_com_apply.
// Each thread sums its particles' terms (mod 2^64) for one galaxy ag in
// registers (a particle of another galaxy first sends the running sums to
// the block's accumulator row); the warps reduce once, at the end.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1) k_recentre(PartK<T> p, const __grid_constant__ SysK s, CenK *cen,
                                                  long long *part) {
    __shared__ unsigned long long red[PM_MAX_GALAXIES][4];
    if (threadIdx.x < PM_MAX_GALAXIES * 4) (&red[0][0])[threadIdx.x] = 0;
    int ag = -1;
    unsigned long long S[4] = {0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    // U particles per round: all their loads are issued before any is used
    // (volatile loads stay where they are written), so a thread keeps U
    // particles' reads in flight
    constexpr int U = 4;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < p.n; i0 += U * stride) {
        uint32_t f[U];
        int gi[U];
        T x[U], y[U], z[U], m[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = i0 + u * stride;
            f[u] = PM_FLAG_LOST;
            if (i < p.n) {
                f[u] = ld_early(p.flags + i);
                gi[u] = ld_early(p.gal + i);
                x[u] = ld_early(p.x + i); y[u] = ld_early(p.y + i); z[u] = ld_early(p.z + i);
                m[u] = ld_early(p.m + i);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (f[u] & PM_FLAG_LOST) continue;
            int Dx, Dy, Dz;
            long long M;
            const int g = com_contrib(s, cen, gi[u], x[u], y[u], z[u], m[u], M, Dx, Dy, Dz);
            if (g < 0) continue;
            if (g != ag) {
                if (ag >= 0) com_flush(part, ag, S);
                ag = g;
            }
            S[0] += (unsigned long long)M;
            S[1] += (unsigned long long)(M * Dx);
            S[2] += (unsigned long long)(M * Dy);
            S[3] += (unsigned long long)(M * Dz);
        }
    }
    __syncthreads();
    com_warp_add(s, red, ag, S);
    com_write_partials(s, red, part);
}

// Step a8 (+a9): acceleration by Eq. (eqn:diff) on the grids the combination
// rule selects for each galaxy (Sec. 2.1), then
//   MODE 0: leap-frog kick-drift   MODE 1: write acceleration
//   MODE 2: kick only              MODE 3: energy / angular momentum sums
// The FP32 kick-drift fits 48 registers without spilling: five blocks per
// SM hide more of the stencil gathers' latency than four at 64.
template <typename T, int MODE>
__global__ void __launch_bounds__(256, (MODE == 0 && sizeof(T) == 4) ? 5 : 3)
    k_force(PartK<T> p, const __grid_constant__ SysK s, const CenK *cen, T dt, T *ax, T *ay, T *az, double *diag) {
    double dsum[7] = {0, 0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < p.n; b += stride) {
        const long long i = b + threadIdx.x;
        if (i < p.n) {
            // the particle's loads (velocities too) issued before the flag
            // test and the stencil gathers, so their latencies overlap
            const uint32_t f = p.flags[i];
            const T xT = p.x[i], yT = p.y[i], zT = p.z[i];
            T v0[3] = {0, 0, 0};
            if (MODE == 0 || MODE == 2) { v0[0] = p.vx[i]; v0[1] = p.vy[i]; v0[2] = p.vz[i]; }
            if (f & PM_FLAG_LOST) {
                if (MODE == 1) { ax[i] = 0; ay[i] = 0; az[i] = 0; }
            } else {
                const float sx = pm_canon(xT, s.sc[0], s.sc_hi[0], s.sc_lo[0]);
                const float sy = pm_canon(yT, s.sc[1], s.sc_hi[1], s.sc_lo[1]);
                const float sz = pm_canon(zT, s.sc[2], s.sc_hi[2], s.sc_lo[2]);
                const T rsx = rel_off(xT, s.sc[0], s.sc_hi[0], s.sc_lo[0]);
                const T rsy = rel_off(yT, s.sc[1], s.sc_hi[1], s.sc_lo[1]);
                const T rsz = rel_off(zT, s.sc[2], s.sc_hi[2], s.sc_lo[2]);
                T acc[3] = {0, 0, 0};
                T phiv = 0;
                T *php = (MODE == 3) ? &phiv : nullptr;
                for (int h = 0; h < s.ngal; ++h) {
                    const GalK &G = s.gal[h];
                    const Cen1 ce = load_cen(cen, h);
                    const float fx = pm_canon(xT, ce.c[0], ce.hi[0], ce.lo[0]);
                    const float fy = pm_canon(yT, ce.c[1], ce.hi[1], ce.lo[1]);
                    const float fz = pm_canon(zT, ce.c[2], ce.hi[2], ce.lo[2]);
                    Cell cf, cm;
                    const int reg = pm_region(G, fx, fy, fz, cf, cm);
                    const Cell cc = pm_cells(G.coarse, sx, sy, sz);
                    if (!cc.ok) continue;  // only after positions changed without a deposit
                    T dx, dy, dz;
                    cell_delta(G.coarse, cc, rsx, rsy, rsz, dx, dy, dz);
                    stencil<T>(G.coarse, static_cast<const T *>(reg == REG_OUTER ? G.phi_call : G.phi_c5), nullptr,
                               cc, dx, dy, dz, acc, php);
                    if (reg != REG_OUTER) {
                        const T rx = rel_off(xT, ce.c[0], ce.hi[0], ce.lo[0]);
                        const T ry = rel_off(yT, ce.c[1], ce.hi[1], ce.lo[1]);
                        const T rz = rel_off(zT, ce.c[2], ce.hi[2], ce.lo[2]);
                        cell_delta(G.med, cm, rx, ry, rz, dx, dy, dz);
                        stencil<T>(G.med, static_cast<const T *>(reg == REG_SHELL ? G.phi_m23 : G.phi_m3), nullptr,
                                   cm, dx, dy, dz, acc, php);
                        if (reg == REG_CORE) {
                            cell_delta(G.fine, cf, rx, ry, rz, dx, dy, dz);
                            if (MODE != 3 && G.fd_x)   // forces from the difference fields
                                stencil_diff<T>(G.fine, static_cast<const T *>(G.fd_x), static_cast<const T *>(G.fd_y),
                                                static_cast<const T *>(G.fd_z), cf, dx, dy, dz, acc);
                            else
                                stencil<T>(G.fine, static_cast<const T *>(G.phi_fine), nullptr, cf, dx, dy, dz, acc,
                                           php);
                        }
                    }
                }
                if (MODE == 0) {
                    const T vx = v0[0] + dt * acc[0], vy = v0[1] + dt * acc[1], vz = v0[2] + dt * acc[2];
                    p.vx[i] = vx; p.vy[i] = vy; p.vz[i] = vz;
                    p.x[i] = xT + dt * vx; p.y[i] = yT + dt * vy; p.z[i] = zT + dt * vz;
                } else if (MODE == 1) {
                    ax[i] = acc[0]; ay[i] = acc[1]; az[i] = acc[2];
                } else if (MODE == 2) {
                    p.vx[i] = v0[0] + dt * acc[0]; p.vy[i] = v0[1] + dt * acc[1]; p.vz[i] = v0[2] + dt * acc[2];
                } else {
                    const double x = (double)xT, y = (double)yT, z = (double)zT;
                    const double hdt = 0.5 * (double)dt;
                    const double vx = (double)p.vx[i] + hdt * (double)acc[0];
                    const double vy = (double)p.vy[i] + hdt * (double)acc[1];
                    const double vz = (double)p.vz[i] + hdt * (double)acc[2];
                    const double m = (double)p.m[i];
                    dsum[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
                    dsum[1] += -0.5 * m * (double)phiv;
                    dsum[3] += m * (y * vz - z * vy);
                    dsum[4] += m * (z * vx - x * vz);
                    dsum[5] += m * (x * vy - y * vx);
                    dsum[6] += 1.0;
                }
            }
        }
    }
    if (MODE == 3) {
        dsum[2] = dsum[0] + dsum[1];
        __shared__ double dred[8][7];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const double v = warp_sum(dsum[k]);
            if (lane == 0) dred[w][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            double v = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += dred[k][threadIdx.x];
            atomicAdd(diag + threadIdx.x, v);
        }
    }
}

// ---------------------------------------------------------------------------
// Spatial counting sort of the particles: key = (galaxy, region, bin of the
// finest grid of that region); a warp then works on particles of the same or
// neighbouring cells, so the deposit atomics and stencil gathers of its lanes
// share addresses.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sort_key(PartK<T> p, const __grid_constant__ SysK s, const CenK *cen,
                                                  SortK so, unsigned *count, unsigned *key, unsigned *rank) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    unsigned k = (unsigned)(so.nkeys - 1);  // lost
    const int g = p.gal[i];
    if (!(p.flags[i] & PM_FLAG_LOST) && g >= 0 && g < s.ngal) {
        const T x = p.x[i], y = p.y[i], z = p.z[i];
        const GalK &G = s.gal[g];
        const Cen1 ce = load_cen(cen, g);
        const float fx = pm_canon(x, ce.c[0], ce.hi[0], ce.lo[0]);
        const float fy = pm_canon(y, ce.c[1], ce.hi[1], ce.lo[1]);
        const float fz = pm_canon(z, ce.c[2], ce.hi[2], ce.lo[2]);
        Cell cf, cm;
        const int reg = pm_region(G, fx, fy, fz, cf, cm);
        const GeomK *gm;
        Cell c;
        if (reg == REG_CORE) { gm = &G.fine; c = cf; }
        else if (reg == REG_SHELL) { gm = &G.med; c = cm; }
        else {
            gm = &G.coarse;
            c = pm_cells(G.coarse, pm_canon(x, s.sc[0], s.sc_hi[0], s.sc_lo[0]),
                         pm_canon(y, s.sc[1], s.sc_hi[1], s.sc_lo[1]), pm_canon(z, s.sc[2], s.sc_hi[2], s.sc_lo[2]));
        }
        if (c.ok) {
            const int b = so.shift[g][reg];
            const long long bin = ((long long)(c.k >> b) * (gm->ny >> b) + (c.j >> b)) * (gm->nx >> b) + (c.i >> b);
            k = (unsigned)(so.base[g][reg] + bin);
        }
    }
    key[i] = k;
    // warp-aggregated ranking: lanes with the same key take consecutive ranks
    // from one atomic (lanes past the end have returned: use the lanes here)
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, k);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(count + k, (unsigned)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[i] = base + __popc(peers & ((1u << lane) - 1u));
}

constexpr int SCAN_TILE = 2048;  // 256 threads x 8

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *tmp, unsigned &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < nw ? tmp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) tmp[lane] = t;
    }
    __syncthreads();
    total = tmp[nw - 1];
    const unsigned before = w > 0 ? tmp[w - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

static __global__ void __launch_bounds__(256) k_scan_reduce(const unsigned *a, long long n, unsigned *bsum) {
    __shared__ unsigned tmp[32];
    const long long t0 = (long long)blockIdx.x * SCAN_TILE;
    unsigned v = 0;
    for (int k = 0; k < SCAN_TILE / 256; ++k) {
        const long long i = t0 + k * 256 + threadIdx.x;
        if (i < n) v += a[i];
    }
    unsigned total;
    block_excl_scan(v, tmp, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

static __global__ void __launch_bounds__(1024) k_scan_top(unsigned *bsum, int nb) {
    __shared__ unsigned tmp[32];
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    unsigned v = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) v += bsum[b0 + k];
    unsigned total;
    unsigned run = block_excl_scan(v, tmp, total);
    for (int k = 0; k < per; ++k)
        if (b0 + k < nb) {
            const unsigned t = bsum[b0 + k];
            bsum[b0 + k] = run;
            run += t;
        }
}

// The count array is allocated with a multiple of SCAN_TILE elements, so a
// thread's eight values are two aligned uint4.
static __global__ void __launch_bounds__(256) k_scan_down(unsigned *a, long long n, const unsigned *bsum) {
    __shared__ unsigned tmp[32];
    const long long t0 = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * (SCAN_TILE / 256);
    uint4 *a4 = reinterpret_cast<uint4 *>(a + t0);
    uint4 u0 = a4[0], u1 = a4[1];
    unsigned v[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    unsigned sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (t0 + k >= n) v[k] = 0u;
        sum += v[k];
    }
    unsigned total;
    unsigned run = block_excl_scan(sum, tmp, total) + bsum[blockIdx.x];
    unsigned o[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { o[k] = run; run += v[k]; }
    a4[0] = make_uint4(o[0], o[1], o[2], o[3]);
    a4[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

// One particle per thread (full grid): every load is issued before the
// destination is known, so a warp keeps all its reads in flight.
// Copies the nine particle arrays (7 of T, 2 of 32-bit ints) from src to
// dst, n elements each.
template <typename T>
__global__ void __launch_bounds__(256) k_copy_particles(PartK<T> src, PartK<T> dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= src.n) return;
    dst.x[i] = src.x[i]; dst.y[i] = src.y[i]; dst.z[i] = src.z[i];
    dst.vx[i] = src.vx[i]; dst.vy[i] = src.vy[i]; dst.vz[i] = src.vz[i];
    const_cast<T *>(dst.m)[i] = src.m[i];
    const_cast<int32_t *>(dst.gal)[i] = src.gal[i];
    dst.flags[i] = src.flags[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_sort_scatter(PartK<T> p, PartK<T> d, const unsigned *key, const unsigned *rank,
                                                      const unsigned *off, long long *perm) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const unsigned k = key[i], r = rank[i];
    const T x = p.x[i], y = p.y[i], z = p.z[i], vx = p.vx[i], vy = p.vy[i], vz = p.vz[i], m = p.m[i];
    const int32_t g = p.gal[i];
    const uint32_t f = p.flags[i];
    const long long j = (long long)off[k] + r;
    d.x[j] = x; d.y[j] = y; d.z[j] = z;
    d.vx[j] = vx; d.vy[j] = vy; d.vz[j] = vz;
    const_cast<T *>(d.m)[j] = m;
    const_cast<int32_t *>(d.gal)[j] = g;
    d.flags[j] = f;
    if (perm) perm[j] = i;
}

template <typename T>
__global__ void k_count_lost(PartK<T> p, unsigned long long *out) {
    unsigned long long c = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride)
        c += (p.flags[i] & PM_FLAG_LOST) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

template <typename T, int L>
__global__ void k_store_hhat(const double *oct, T *out, int nx, int ny, double scale) {
    constexpr int NS = nstages(L), RL = radix(L, NS - 1, false), HS = pm_hhat_stride(L);
    const long long ncol = (long long)(nx + 1) * (ny + 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncol * HS;
         i += (long long)gridDim.x * blockDim.x) {
        const long long col = i / HS;
        const int w = (int)(i % HS);
        int kzr;
        if (hhat_thread_major(L)) {   // register w % 16 of thread w / 16
            const int e = w % E, t = w / E;
            const int kz = pmfft::in_row<L, NS - 1, false>(t, e / RL, e % RL);
            kzr = kz <= L / 2 ? kz : L - kz;
        } else {
            kzr = w;                  // padding beyond nz = L/2
        }
        out[i] = kzr <= L / 2 ? (T)(oct[(long long)kzr * ncol + col] * scale) : (T)0;
    }
}

}  // namespace pmk

// ---------------------------------------------------------------------------
// Host launchers (explicitly instantiated per precision)
// ---------------------------------------------------------------------------
namespace pmk_host {

// One particle per thread up to 2^16 blocks (16.7M particles); larger sets
// loop (grid-stride).
inline int particle_grid(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 1LL << 16;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename T, int L, int MODE> int col_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pmk::k_col<T, L, MODE>, pmk::CShape<T, L>::THREADS,
                                                          pmk::col_smem<T, L, MODE>()) != cudaSuccess || nb < 1)
            nb = 1;
        cached = nb;
    }
    return cached;
}

template <typename T, int L, int DM> int colw_blocks_per_sm() {
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pmk::k_colw<T, L, DM>, pmk::WShape<T, L>::THREADS,
                                                          pmk::colw_smem<T, L>()) != cudaSuccess || nb < 1)
            nb = 1;
        cached = nb;
    }
    return cached;
}

inline int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    }
    return n;
}

template <typename T, int L> cudaError_t attrs_L() {
    cudaError_t e;
    e = cudaFuncSetAttribute(pmk::k_col<T, L, COL_YFWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pmk::col_smem<T, L, COL_YFWD>());
    if (e) return e;
    e = cudaFuncSetAttribute(pmk::k_colw<T, L, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pmk::colw_smem<T, L>());
    if (e) return e;
    e = cudaFuncSetAttribute(pmk::k_colw<T, L, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pmk::colw_smem<T, L>());
    if (e) return e;
    if constexpr (L <= 256) {
        e = cudaFuncSetAttribute(pmk::k_colw<T, L, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pmk::colw_smem<T, L>());
        if (e) return e;
    }
    e = cudaFuncSetAttribute(pmk::k_col<T, L, COL_YINV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pmk::col_smem<T, L, COL_YINV>());
    if (e) return e;
    e = cudaFuncSetAttribute(pmk::k_xfwd<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pmk::xpass_smem<T, L>());
    if (e) return e;
    return cudaFuncSetAttribute(pmk::k_xinv<T, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pmk::xpass_smem<T, L>());
}

// Persistent x passes: one wave of blocks (occupancy x SMs), each walking
// groups of rows.
template <typename K> int resident_blocks(K kernel, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}
// Launch with programmatic stream serialisation (the FFT passes of a chain:
// each waits for its predecessor with griddepcontrol.wait after its
// prologue).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

inline int ilog2(long long v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}
template <typename T, int L> cudaError_t xfwd_L(PassBatch b, cudaStream_t st) {
    static int nb = resident_blocks(pmk::k_xfwd<T, L>, pmk::NT, pmk::xpass_smem<T, L>());
    const long long gpi = std::max(1LL, (long long)b.a[0].ny * b.a[0].nz / pmk::XShape<L>::LINES);
    b.lgi = ilog2(gpi);
    const long long grid = std::min((long long)b.n << b.lgi, (long long)nb * num_sms());
    return launch_pdl(pmk::k_xfwd<T, L>, (unsigned)grid, pmk::NT, pmk::xpass_smem<T, L>(), st, b);
}
template <typename T, int L> cudaError_t xinv_L(PassBatch b, cudaStream_t st) {
    static int nb = resident_blocks(pmk::k_xinv<T, L>, pmk::NT, pmk::xpass_smem<T, L>());
    const long long gpi = std::max(1LL, (long long)b.a[0].ny * b.a[0].nz / pmk::XShape<L>::LINES);
    b.lgi = ilog2(gpi);
    const long long grid = std::min((long long)b.n << b.lgi, (long long)nb * num_sms());
    return launch_pdl(pmk::k_xinv<T, L>, (unsigned)grid, pmk::NT, pmk::xpass_smem<T, L>(), st, b);
}
template <typename T, int L, int MODE> cudaError_t col_LM(PassBatch b, cudaStream_t st) {
    constexpr int COLS = pmk::CShape<T, L>::COLS;
    b.lgi = ilog2((long long)b.a[0].nz * ((2 * b.a[0].nx + COLS - 1) / COLS));
    const long long ntiles = (long long)b.n << b.lgi;
    long long grid = (long long)col_blocks_per_sm<T, L, MODE>() * num_sms();
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    return launch_pdl(pmk::k_col<T, L, MODE>, (unsigned)grid, pmk::CShape<T, L>::THREADS,
                      pmk::col_smem<T, L, MODE>(), st, b);
}
template <typename T, int L> cudaError_t zconv_L(PassBatch b, cudaStream_t st) {
    typedef pmk::WShape<T, L> S;
    b.lgi = ilog2(((long long)4 * b.a[0].ny * b.a[0].nx) / S::COLS);   // COLS divides the 2ny x 2nx columns
    const long long ntiles = (long long)b.n << b.lgi;
    const bool dm = b.a[0].dmode != 0;
    if constexpr (L <= 256) {
        if (b.a[0].dmode == 3) {   // both difference fields in one pass (see PairArgs)
            long long g2 = (long long)colw_blocks_per_sm<T, L, 2>() * num_sms();
            if (g2 > ntiles) g2 = ntiles;
            if (g2 < 1) g2 = 1;
            return launch_pdl(pmk::k_colw<T, L, 2>, (unsigned)g2, S::THREADS, pmk::colw_smem<T, L>(), st, b);
        }
    }
    if (b.a[0].dmode == 3) return cudaErrorInvalidValue;
    long long grid = (long long)(dm ? colw_blocks_per_sm<T, L, 1>() : colw_blocks_per_sm<T, L, 0>()) * num_sms();
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    if (dm) return launch_pdl(pmk::k_colw<T, L, 1>, (unsigned)grid, S::THREADS, pmk::colw_smem<T, L>(), st, b);
    return launch_pdl(pmk::k_colw<T, L, 0>, (unsigned)grid, S::THREADS, pmk::colw_smem<T, L>(), st, b);
}
template <typename T, int L> cudaError_t col_L(const PassBatch &b, int mode, cudaStream_t st) {
    if (mode == COL_YFWD) return col_LM<T, L, COL_YFWD>(b, st);
    if (mode == COL_ZCONV) return zconv_L<T, L>(b, st);
    return col_LM<T, L, COL_YINV>(b, st);
}

#define PM_SWITCH_L(L, CALL)                          \
    switch (L) {                                      \
        case 16: return CALL(16);                     \
        case 32: return CALL(32);                     \
        case 64: return CALL(64);                     \
        case 128: return CALL(128);                   \
        case 256: return CALL(256);                   \
        case 512: return CALL(512);                   \
        default: return cudaErrorInvalidValue;        \
    }

}  // namespace pmk_host

template <typename T> cudaError_t pm_set_attrs() {
    cudaError_t e;
    if ((e = pmk_host::attrs_L<T, 16>())) return e;
    if ((e = pmk_host::attrs_L<T, 32>())) return e;
    if ((e = pmk_host::attrs_L<T, 64>())) return e;
    if ((e = pmk_host::attrs_L<T, 128>())) return e;
    if ((e = pmk_host::attrs_L<T, 256>())) return e;
    return pmk_host::attrs_L<T, 512>();
}

template <typename T> cudaError_t pm_launch_xfwd(PassBatch b, cudaStream_t st) {
    if (b.n < 1 || b.n > PM_BATCH) return cudaErrorInvalidValue;
#define PM_XF(LL) pmk_host::xfwd_L<T, LL>(b, st)
    PM_SWITCH_L(2 * b.a[0].nx, PM_XF)
#undef PM_XF
}
template <typename T> cudaError_t pm_launch_xinv(PassBatch b, cudaStream_t st) {
    if (b.n < 1 || b.n > PM_BATCH) return cudaErrorInvalidValue;
#define PM_XI(LL) pmk_host::xinv_L<T, LL>(b, st)
    PM_SWITCH_L(2 * b.a[0].nx, PM_XI)
#undef PM_XI
}
template <typename T> cudaError_t pm_launch_col(PassBatch b, int mode, cudaStream_t st) {
    if (b.n < 1 || b.n > PM_BATCH) return cudaErrorInvalidValue;
    const int L = (mode == COL_ZCONV) ? 2 * b.a[0].nz : 2 * b.a[0].ny;
#define PM_CO(LL) pmk_host::col_L<T, LL>(b, mode, st)
    PM_SWITCH_L(L, PM_CO)
#undef PM_CO
}

template <typename T>
cudaError_t pm_launch_deposit(const PartK<T> &p, const SysK &sk, const CenK *cen, int aggregate, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    pmk::k_deposit<T><<<pmk_host::particle_grid(p.n), 256, 0, st>>>(p, sk, cen, aggregate);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_force(int mode, const PartK<T> &p, const SysK &sk, const CenK *cen, double dt,
                            T *ax, T *ay, T *az, double *diag, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    const int g = pmk_host::particle_grid(p.n);
    switch (mode) {
        case 0: pmk::k_force<T, 0><<<g, 256, 0, st>>>(p, sk, cen, (T)dt, ax, ay, az, diag); break;
        case 1: pmk::k_force<T, 1><<<g, 256, 0, st>>>(p, sk, cen, (T)dt, ax, ay, az, diag); break;
        case 2: pmk::k_force<T, 2><<<g, 256, 0, st>>>(p, sk, cen, (T)dt, ax, ay, az, diag); break;
        case 3: pmk::k_force<T, 3><<<g, 256, 0, st>>>(p, sk, cen, (T)dt, ax, ay, az, diag); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_recentre(const PartK<T> &p, const SysK &sk, CenK *cen, long long *part, int phase,
                               cudaStream_t st) {
    if ((phase & 1) && p.n > 0) {
        // one full wave of resident blocks (5 per SM in FP32, 48 registers
        // for four particles' loads in flight): each thread sums several
        // particles in registers before the one warp reduction
        static int bps = 0;
        if (!bps && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pmk::k_recentre<T>, 256, 0) != cudaSuccess ||
                     bps < 1))
            bps = 1;
        const int g = std::min(pmk_host::particle_grid(p.n), bps * pmk_host::num_sms());
        pmk::k_recentre<T><<<g, 256, 0, st>>>(p, sk, cen, part);
    }
    if (phase & 2) pmk::k_com_apply<<<1, 256, 0, st>>>(sk, part, cen);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_sort(const PartK<T> &p, const PartK<T> &scratch, const SysK &sk, const CenK *cen,
                           const SortK &so, unsigned *count, unsigned *key, unsigned *rank, unsigned *bsum,
                           long long *perm, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)so.nkeys * sizeof(unsigned), st);
    if (e) return e;
    const unsigned g = (unsigned)((p.n + 255) / 256);
    pmk::k_sort_key<T><<<g, 256, 0, st>>>(p, sk, cen, so, count, key, rank);
    const int nb = (int)((so.nkeys + pmk::SCAN_TILE - 1) / pmk::SCAN_TILE);
    pmk::k_scan_reduce<<<nb, 256, 0, st>>>(count, so.nkeys, bsum);
    pmk::k_scan_top<<<1, 1024, 0, st>>>(bsum, nb);
    pmk::k_scan_down<<<nb, 256, 0, st>>>(count, so.nkeys, bsum);
    pmk::k_sort_scatter<T><<<g, 256, 0, st>>>(p, scratch, key, rank, count, perm);
    if ((e = cudaGetLastError())) return e;
    PartK<T> sc = scratch;
    sc.n = p.n;
    pmk::k_copy_particles<T><<<g, 256, 0, st>>>(sc, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_count_lost(const PartK<T> &p, unsigned long long *out, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    pmk::k_count_lost<T><<<pmk_host::particle_grid(p.n), 256, 0, st>>>(p, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_store_hhat(const double *oct, T *out, int nx, int ny, int nz, double scale, cudaStream_t st) {
    const int g = pmk_host::particle_grid(pm_hhat_table_size(nx, ny, nz));
#define PM_SH(LL) (pmk::k_store_hhat<T, LL><<<g, 256, 0, st>>>(oct, out, nx, ny, scale), cudaGetLastError())
    PM_SWITCH_L(2 * nz, PM_SH)
#undef PM_SH
}

#define PM_INSTANTIATE(T)                                                                                       \
    template cudaError_t pm_set_attrs<T>();                                                                    \
    template cudaError_t pm_launch_xfwd<T>(PassBatch, cudaStream_t);                                          \
    template cudaError_t pm_launch_xinv<T>(PassBatch, cudaStream_t);                                          \
    template cudaError_t pm_launch_col<T>(PassBatch, int, cudaStream_t);                                      \
    template cudaError_t pm_launch_deposit<T>(const PartK<T> &, const SysK &, const CenK *, int, cudaStream_t); \
    template cudaError_t pm_launch_force<T>(int, const PartK<T> &, const SysK &, const CenK *, double, T *, T *, \
                                            T *, double *, cudaStream_t);                                      \
    template cudaError_t pm_launch_recentre<T>(const PartK<T> &, const SysK &, CenK *, long long *, int,       \
                                               cudaStream_t);                                                  \
    template cudaError_t pm_launch_count_lost<T>(const PartK<T> &, unsigned long long *, cudaStream_t);       \
    template cudaError_t pm_launch_sort<T>(const PartK<T> &, const PartK<T> &, const SysK &, const CenK *,     \
                                           const SortK &, unsigned *, unsigned *, unsigned *, unsigned *,       \
                                           long long *, cudaStream_t);                                          \
    template cudaError_t pm_store_hhat<T>(const double *, T *, int, int, int, double, cudaStream_t);
