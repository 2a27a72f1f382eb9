// Cloud-in-cell (CIC) variant of the step and its adjoint, for differentiable
// runs.  The paper's nearest-grid-point assignment (Eq. eqn:cell) has zero
// position gradient almost everywhere; this variant spreads each mass over
// the 8 cells around it with trilinear weights W, takes the grid field as
// the central difference of the potential (first term of Eq. eqn:diff) and
// interpolates it back with the same weights.  Regions, mass sets, the
// doubled-grid convolution and the combination rule of Sec. 2.1 are those of
// the NGP step; grid centres are held fixed.
//
// CIC cells: the NGP cell a of Eq. (eqn:cell) (canonical rounding) fixes the
// particle; t = Delta / l in [-1/2, 1/2] is its offset from that cell's
// centre; the lower CIC cell is a - 1 with fraction t + 1 when t < 0, else a
// with fraction t.  With a in the usable box 2..N-3 the CIC cells and their
// difference neighbours stay inside 0..N-1.
//
// Adjoint (vector-Jacobian product of the acceleration a(x, m) with a
// cotangent u per particle), with K the symmetric convolution and D the
// central difference (D^T = -D on the grid):
//   direct term  dx_i += sum_c grad W(x_i - x_c) (g[c] . u_i)
//   field term   lam_k = K sum_d D_d^T psi_k^d, psi_k^d = sum_i W u_i^d over the
//                field points that read set k; then for each particle j of mass
//                set k: dx_j += m_j sum_c grad W lam_k[c], dm_j += sum_c W lam_k[c].
// The sum_d D_d^T psi is spread directly from each particle (32 cells) as
// int64 fixed point, so the adjoint solve reuses the FFT passes unchanged.
// Pair slots are loaded so that the solver's stored outputs are the lam_k
// the mass sets need: medium a = psi_2 - psi_3, b = psi_3 (outputs
// lam_2 = a + b, lam_3 = b); coarse a = psi_4 - psi_5, b = psi_5.
#pragma once

#include "pm_particle.cuh"

namespace pmk {

template <typename T> struct Cic {
    size_t base;          // offset of the lower cell (a0, b0, c0)
    T w[3][2];            // per axis: weights of the lower and upper cell
    T il[3];              // 1 / l per axis
};

template <typename T>
__device__ __forceinline__ Cic<T> cic_cell(const GeomK &g, const Cell &cl, T rx, T ry, T rz) {
    T d[3];
    cell_delta(g, cl, rx, ry, rz, d[0], d[1], d[2]);
    Cic<T> c;
    c.il[0] = c.il[1] = pick<T>(2.0 * g.c_gx, g.fil_xy);
    c.il[2] = pick<T>(2.0 * g.c_gz, g.fil_z);
    int idx[3] = {cl.i, cl.j, cl.k};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T t = d[a] * c.il[a];
        if (t < (T)0) { idx[a] -= 1; t += (T)1; }
        c.w[a][0] = (T)1 - t;
        c.w[a][1] = t;
    }
    c.base = ((size_t)idx[2] * g.ny + idx[1]) * g.nx + idx[0];
    return c;
}

// Central-difference field of F at the 8 CIC cells: gr[dk][dj][di][axis].
template <typename T>
__device__ __forceinline__ void cic_grad8(const GeomK &g, const T *__restrict__ F, const Cic<T> &c,
                                          T gr[2][2][2][3]) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    const T *b = F + c.base;
    auto ld = [&](int di, int dj, int dk) -> T { return __ldg(b + di + dj * sy + dk * sz); };
    T cen[2][2][2];
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) cen[dk][dj][di] = ld(di, dj, dk);
    const T hx = c.il[0] * (T)0.5, hz = c.il[2] * (T)0.5;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            const T lo = ld(-1, dj, dk), hi = ld(2, dj, dk);
            gr[dk][dj][0][0] = (cen[dk][dj][1] - lo) * hx;
            gr[dk][dj][1][0] = (hi - cen[dk][dj][0]) * hx;
        }
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            const T lo = ld(di, -1, dk), hi = ld(di, 2, dk);
            gr[dk][0][di][1] = (cen[dk][1][di] - lo) * hx;
            gr[dk][1][di][1] = (hi - cen[dk][0][di]) * hx;
        }
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            const T lo = ld(di, dj, -1), hi = ld(di, dj, 2);
            gr[0][dj][di][2] = (cen[1][dj][di] - lo) * hz;
            gr[1][dj][di][2] = (hi - cen[0][dj][di]) * hz;
        }
}

// acc += sum_c W g_c   (VJP == false)
// gx  += sum_c grad W (g_c . u)   (VJP == true)
template <typename T, bool VJP>
__device__ __forceinline__ void cic_field(const GeomK &g, const void *F, const Cic<T> &c, const T *u, T *out) {
    T gr[2][2][2][3];
    cic_grad8<T>(g, static_cast<const T *>(F), c, gr);
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const T *v = gr[dk][dj][di];
                if (!VJP) {
                    const T W = c.w[0][di] * c.w[1][dj] * c.w[2][dk];
                    out[0] += W * v[0];
                    out[1] += W * v[1];
                    out[2] += W * v[2];
                } else {
                    const T s = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
                    out[0] += (di ? c.il[0] : -c.il[0]) * c.w[1][dj] * c.w[2][dk] * s;
                    out[1] += (dj ? c.il[1] : -c.il[1]) * c.w[0][di] * c.w[2][dk] * s;
                    out[2] += (dk ? c.il[2] : -c.il[2]) * c.w[0][di] * c.w[1][dj] * s;
                }
            }
}

// lam_w += sum_c W F_c, lam_g += sum_c grad W F_c (the 8 CIC cells).
template <typename T>
__device__ __forceinline__ void cic_gather(const GeomK &g, const void *Fv, const Cic<T> &c, T &lw, T *lg) {
    const T *F = static_cast<const T *>(Fv) + c.base;
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const T f = __ldg(F + di + dj * sy + dk * sz);
                lw += c.w[0][di] * c.w[1][dj] * c.w[2][dk] * f;
                lg[0] += (di ? c.il[0] : -c.il[0]) * c.w[1][dj] * c.w[2][dk] * f;
                lg[1] += (dj ? c.il[1] : -c.il[1]) * c.w[0][di] * c.w[2][dk] * f;
                lg[2] += (dk ? c.il[2] : -c.il[2]) * c.w[0][di] * c.w[1][dj] * f;
            }
}

__device__ __forceinline__ long long cic_q(float v, float s) { return __float2ll_rn(v * s); }
__device__ __forceinline__ long long cic_q(double v, double s) { return __double2ll_rn(v * s); }

// Forward deposit: m W into the 8 cells (fixed point, scale qs = 2^s).
template <typename T>
__device__ __forceinline__ void cic_spread_mass(const GeomK &g, unsigned long long *rho, const Cic<T> &c, T m, T qs) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    unsigned long long *b = rho + c.base;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const T W = c.w[0][di] * c.w[1][dj] * c.w[2][dk];
                atomicAdd(b + di + dj * sy + dk * sz, (unsigned long long)cic_q(m * W, qs));
            }
}

// Adjoint spread: sign * sum_d D_d^T (W u_d) into the 32 cells it touches
// (fixed point, scale qs).  h[d] = u_d / (2 l_d).
template <typename T>
__device__ __forceinline__ void cic_spread_adj(const GeomK &g, unsigned long long *rho, const Cic<T> &c, const T *h,
                                               T qs) {
    const long long sy = g.nx, sz = (long long)g.nx * g.ny;
    unsigned long long *b = rho + c.base;
    auto add = [&](int di, int dj, int dk, T v) {
        atomicAdd(b + di + dj * sy + dk * sz, (unsigned long long)cic_q(v, qs));
    };
    const T(&w)[3][2] = c.w;
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const T vx = h[0] * w[1][dj] * w[2][dk] * (di ? w[0][0] : -w[0][1]);
                const T vy = h[1] * w[0][di] * w[2][dk] * (dj ? w[1][0] : -w[1][1]);
                const T vz = h[2] * w[0][di] * w[1][dj] * (dk ? w[2][0] : -w[2][1]);
                add(di, dj, dk, vx + vy + vz);
            }
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            add(-1, dj, dk, -h[0] * w[0][0] * w[1][dj] * w[2][dk]);
            add(2, dj, dk, h[0] * w[0][1] * w[1][dj] * w[2][dk]);
        }
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            add(di, -1, dk, -h[1] * w[1][0] * w[0][di] * w[2][dk]);
            add(di, 2, dk, h[1] * w[1][1] * w[0][di] * w[2][dk]);
        }
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            add(di, dj, -1, -h[2] * w[2][0] * w[0][di] * w[1][dj]);
            add(di, dj, 2, h[2] * w[2][1] * w[0][di] * w[1][dj]);
        }
}

// Particle position relative to the system centre and to galaxy h's centre.
template <typename T> struct Rel {
    float sx, sy, sz;   // canonical FP32 offsets from the system centre (cells, lost test)
    T rsx, rsy, rsz;    // offsets from the system centre (Delta)
};
template <typename T>
__device__ __forceinline__ Rel<T> rel_sys(const SysK &s, T x, T y, T z) {
    Rel<T> r;
    r.sx = pm_canon(x, s.sc[0], s.sc_hi[0], s.sc_lo[0]);
    r.sy = pm_canon(y, s.sc[1], s.sc_hi[1], s.sc_lo[1]);
    r.sz = pm_canon(z, s.sc[2], s.sc_hi[2], s.sc_lo[2]);
    r.rsx = rel_off(x, s.sc[0], s.sc_hi[0], s.sc_lo[0]);
    r.rsy = rel_off(y, s.sc[1], s.sc_hi[1], s.sc_lo[1]);
    r.rsz = rel_off(z, s.sc[2], s.sc_hi[2], s.sc_lo[2]);
    return r;
}

// Forward CIC deposit with the lost test and mass sets of the NGP deposit.
template <typename T>
__global__ void __launch_bounds__(256) k_cic_deposit(PartK<T> p, const __grid_constant__ SysK s, const CenK *cen) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        const uint32_t f = p.flags[i];
        if (f & PM_FLAG_LOST) continue;
        const T x = p.x[i], y = p.y[i], z = p.z[i];
        const int g = p.gal[i];
        const Rel<T> rs = rel_sys(s, x, y, z);
        bool lost = !(pm_r2(rs.sx, rs.sy, rs.sz) < s.rsys2);
        if (g < 0 || g >= s.ngal) lost = true;
        Cell cc;
        cc.i = cc.j = cc.k = 0; cc.ok = false;
        for (int h = 0; h < s.ngal; ++h) {
            const Cell ch = pm_cells(s.gal[h].coarse, rs.sx, rs.sy, rs.sz);
            lost = lost || !ch.ok;
            if (h == g) cc = ch;
        }
        if (lost) { p.flags[i] = f | PM_FLAG_LOST; continue; }
        const GalK &G = s.gal[g];
        const Cen1 ce = load_cen(cen, g);
        Cell cf, cm;
        const int reg = pm_region(G, pm_canon(x, ce.c[0], ce.hi[0], ce.lo[0]), pm_canon(y, ce.c[1], ce.hi[1], ce.lo[1]),
                                  pm_canon(z, ce.c[2], ce.hi[2], ce.lo[2]), cf, cm);
        const T m = p.m[i], qs = pick<T>(s.mscale, s.mscale_f);
        const Cic<T> kc = cic_cell<T>(G.coarse, cc, rs.rsx, rs.rsy, rs.rsz);
        if (reg == REG_OUTER) {
            cic_spread_mass<T>(G.coarse, G.rho[4], kc, m, qs);
            continue;
        }
        const T rx = rel_off(x, ce.c[0], ce.hi[0], ce.lo[0]);
        const T ry = rel_off(y, ce.c[1], ce.hi[1], ce.lo[1]);
        const T rz = rel_off(z, ce.c[2], ce.hi[2], ce.lo[2]);
        cic_spread_mass<T>(G.coarse, G.rho[3], kc, m, qs);
        const Cic<T> km = cic_cell<T>(G.med, cm, rx, ry, rz);
        if (reg == REG_CORE) {
            cic_spread_mass<T>(G.med, G.rho[1], km, m, qs);
            cic_spread_mass<T>(G.fine, G.rho[0], cic_cell<T>(G.fine, cf, rx, ry, rz), m, qs);
        } else {
            cic_spread_mass<T>(G.med, G.rho[2], km, m, qs);
        }
    }
}

// Field-point kernels over every galaxy's grids (combination rule):
//   MODE 0: v += dtk a, x += dtd v     MODE 1: write a
//   MODE 2: g += u^T (d a / d x_i) direct term (positions' own weights)
//   MODE 3: adjoint spread of u into the pair slots (scale qs)
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_cic_field(PartK<T> p, const __grid_constant__ SysK s, const CenK *cen,
                                                   T dtk, T dtd, T *ox, T *oy, T *oz, const T *ux, const T *uy,
                                                   const T *uz, T qs) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        if (p.flags[i] & PM_FLAG_LOST) {
            if (MODE == 1) { ox[i] = 0; oy[i] = 0; oz[i] = 0; }
            continue;
        }
        const T xT = p.x[i], yT = p.y[i], zT = p.z[i];
        const Rel<T> rs = rel_sys(s, xT, yT, zT);
        T u[3] = {0, 0, 0};
        if (MODE >= 2) { u[0] = ux[i]; u[1] = uy[i]; u[2] = uz[i]; }
        T out[3] = {0, 0, 0};
        for (int h = 0; h < s.ngal; ++h) {
            const GalK &G = s.gal[h];
            const Cen1 ce = load_cen(cen, h);
            Cell cf, cm;
            const int reg = pm_region(G, pm_canon(xT, ce.c[0], ce.hi[0], ce.lo[0]),
                                      pm_canon(yT, ce.c[1], ce.hi[1], ce.lo[1]),
                                      pm_canon(zT, ce.c[2], ce.hi[2], ce.lo[2]), cf, cm);
            const Cell cc = pm_cells(G.coarse, rs.sx, rs.sy, rs.sz);
            if (!cc.ok) continue;  // only after positions changed without a deposit
            const Cic<T> kc = cic_cell<T>(G.coarse, cc, rs.rsx, rs.rsy, rs.rsz);
            Cic<T> km, kf;
            if (reg != REG_OUTER) {
                const T rx = rel_off(xT, ce.c[0], ce.hi[0], ce.lo[0]);
                const T ry = rel_off(yT, ce.c[1], ce.hi[1], ce.lo[1]);
                const T rz = rel_off(zT, ce.c[2], ce.hi[2], ce.lo[2]);
                km = cic_cell<T>(G.med, cm, rx, ry, rz);
                if (reg == REG_CORE) kf = cic_cell<T>(G.fine, cf, rx, ry, rz);
            }
            if (MODE == 3) {
                T hp[3] = {u[0] * pick<T>(G.coarse.c_gx, G.coarse.fc_gx), u[1] * pick<T>(G.coarse.c_gx, G.coarse.fc_gx), u[2] * pick<T>(G.coarse.c_gz, G.coarse.fc_gz)};
                T hm[3] = {-hp[0], -hp[1], -hp[2]};
                cic_spread_adj<T>(G.coarse, G.rho[4], kc, hp, qs);         // psi_5 (all points)
                if (reg == REG_OUTER) continue;
                cic_spread_adj<T>(G.coarse, G.rho[3], kc, hm, qs);         // psi_4 - psi_5
                T mp[3] = {u[0] * pick<T>(G.med.c_gx, G.med.fc_gx), u[1] * pick<T>(G.med.c_gx, G.med.fc_gx), u[2] * pick<T>(G.med.c_gz, G.med.fc_gz)};
                cic_spread_adj<T>(G.med, G.rho[2], km, mp, qs);            // psi_3 (core, shell)
                if (reg == REG_CORE) {
                    T mm[3] = {-mp[0], -mp[1], -mp[2]};
                    cic_spread_adj<T>(G.med, G.rho[1], km, mm, qs);        // psi_2 - psi_3
                    T fp[3] = {u[0] * pick<T>(G.fine.c_gx, G.fine.fc_gx), u[1] * pick<T>(G.fine.c_gx, G.fine.fc_gx), u[2] * pick<T>(G.fine.c_gz, G.fine.fc_gz)};
                    cic_spread_adj<T>(G.fine, G.rho[0], kf, fp, qs);       // psi_1
                }
                continue;
            }
            constexpr bool VJP = (MODE == 2);
            cic_field<T, VJP>(G.coarse, reg == REG_OUTER ? G.phi_call : G.phi_c5, kc, u, out);
            if (reg != REG_OUTER) {
                cic_field<T, VJP>(G.med, reg == REG_SHELL ? G.phi_m23 : G.phi_m3, km, u, out);
                if (reg == REG_CORE) cic_field<T, VJP>(G.fine, G.phi_fine, kf, u, out);
            }
        }
        if (MODE == 0) {
            const T vx = p.vx[i] + dtk * out[0], vy = p.vy[i] + dtk * out[1], vz = p.vz[i] + dtk * out[2];
            p.vx[i] = vx; p.vy[i] = vy; p.vz[i] = vz;
            p.x[i] = xT + dtd * vx; p.y[i] = yT + dtd * vy; p.z[i] = zT + dtd * vz;
        } else if (MODE == 1) {
            ox[i] = out[0]; oy[i] = out[1]; oz[i] = out[2];
        } else if (MODE == 2) {
            ox[i] += out[0]; oy[i] += out[1]; oz[i] += out[2];
        }
    }
}

// Field term of the adjoint for each particle's own mass sets: the adjoint
// solve left lam_1 in the fine sum slot, lam_2 (medium sum), lam_3 (medium
// b), lam_4 (coarse sum) and lam_5 (coarse b, or the sum without medium).
template <typename T>
__global__ void __launch_bounds__(256) k_cic_gather(PartK<T> p, const __grid_constant__ SysK s, const CenK *cen,
                                                    T *gx, T *gy, T *gz, T *gm) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        if (p.flags[i] & PM_FLAG_LOST) continue;
        const int g = p.gal[i];
        if (g < 0 || g >= s.ngal) continue;
        const T x = p.x[i], y = p.y[i], z = p.z[i];
        const Rel<T> rs = rel_sys(s, x, y, z);
        const GalK &G = s.gal[g];
        const Cen1 ce = load_cen(cen, g);
        Cell cf, cm;
        const int reg = pm_region(G, pm_canon(x, ce.c[0], ce.hi[0], ce.lo[0]), pm_canon(y, ce.c[1], ce.hi[1], ce.lo[1]),
                                  pm_canon(z, ce.c[2], ce.hi[2], ce.lo[2]), cf, cm);
        const Cell cc = pm_cells(G.coarse, rs.sx, rs.sy, rs.sz);
        if (!cc.ok) continue;
        T lw = 0, lg[3] = {0, 0, 0};
        const Cic<T> kc = cic_cell<T>(G.coarse, cc, rs.rsx, rs.rsy, rs.rsz);
        if (reg == REG_OUTER) {
            cic_gather<T>(G.coarse, G.phi_c5, kc, lw, lg);
        } else {
            const T rx = rel_off(x, ce.c[0], ce.hi[0], ce.lo[0]);
            const T ry = rel_off(y, ce.c[1], ce.hi[1], ce.lo[1]);
            const T rz = rel_off(z, ce.c[2], ce.hi[2], ce.lo[2]);
            cic_gather<T>(G.coarse, G.phi_call, kc, lw, lg);
            const Cic<T> km = cic_cell<T>(G.med, cm, rx, ry, rz);
            if (reg == REG_CORE) {
                cic_gather<T>(G.med, G.phi_m23, km, lw, lg);
                cic_gather<T>(G.fine, G.phi_fine, cic_cell<T>(G.fine, cf, rx, ry, rz), lw, lg);
            } else {
                cic_gather<T>(G.med, G.phi_m3, km, lw, lg);
            }
        }
        const T m = p.m[i];
        gx[i] += m * lg[0];
        gy[i] += m * lg[1];
        gz[i] += m * lg[2];
        gm[i] += lw;
    }
}

// max |u| over live particles (as float bits; non-finite values give +inf).
template <typename T>
__global__ void __launch_bounds__(256) k_cic_umax(PartK<T> p, const T *ux, const T *uy, const T *uz, unsigned *out) {
    float mx = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        if (p.flags[i] & PM_FLAG_LOST) continue;
        const T a = fmax(fabs(ux[i]), fmax(fabs(uy[i]), fabs(uz[i])));
        const float af = (a == a) ? (float)a : __int_as_float(0x7f800000);
        mx = fmaxf(mx, af);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

}  // namespace pmk

// ---------------------------------------------------------------------------
// Host launchers (instantiated for float and double in pm_cic.cu)
// ---------------------------------------------------------------------------
namespace pmk_cic_host {
inline int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < (1LL << 16) ? (b > 0 ? b : 1) : (1LL << 16));
}
}  // namespace pmk_cic_host

template <typename T>
cudaError_t pm_launch_cic_deposit(const PartK<T> &p, const SysK &sk, const CenK *cen, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    pmk::k_cic_deposit<T><<<pmk_cic_host::grid_for(p.n), 256, 0, st>>>(p, sk, cen);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_cic_field(int mode, const PartK<T> &p, const SysK &sk, const CenK *cen, double dtk, double dtd,
                                T *ox, T *oy, T *oz, const T *ux, const T *uy, const T *uz, double qs,
                                cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    const int g = pmk_cic_host::grid_for(p.n);
    switch (mode) {
        case 0: pmk::k_cic_field<T, 0><<<g, 256, 0, st>>>(p, sk, cen, (T)dtk, (T)dtd, ox, oy, oz, ux, uy, uz, (T)qs); break;
        case 1: pmk::k_cic_field<T, 1><<<g, 256, 0, st>>>(p, sk, cen, (T)dtk, (T)dtd, ox, oy, oz, ux, uy, uz, (T)qs); break;
        case 2: pmk::k_cic_field<T, 2><<<g, 256, 0, st>>>(p, sk, cen, (T)dtk, (T)dtd, ox, oy, oz, ux, uy, uz, (T)qs); break;
        case 3: pmk::k_cic_field<T, 3><<<g, 256, 0, st>>>(p, sk, cen, (T)dtk, (T)dtd, ox, oy, oz, ux, uy, uz, (T)qs); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_cic_gather(const PartK<T> &p, const SysK &sk, const CenK *cen, T *gx, T *gy, T *gz, T *gm,
                                 cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    pmk::k_cic_gather<T><<<pmk_cic_host::grid_for(p.n), 256, 0, st>>>(p, sk, cen, gx, gy, gz, gm);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pm_launch_cic_umax(const PartK<T> &p, const T *ux, const T *uy, const T *uz, unsigned *out,
                               cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    pmk::k_cic_umax<T><<<pmk_cic_host::grid_for(p.n), 256, 0, st>>>(p, ux, uy, uz, out);
    return cudaGetLastError();
}

#define PM_CIC_INSTANTIATE(T)                                                                                  \
    template cudaError_t pm_launch_cic_deposit<T>(const PartK<T> &, const SysK &, const CenK *, cudaStream_t); \
    template cudaError_t pm_launch_cic_field<T>(int, const PartK<T> &, const SysK &, const CenK *, double,     \
                                                double, T *, T *, T *, const T *, const T *, const T *, double, \
                                                cudaStream_t);                                                 \
    template cudaError_t pm_launch_cic_gather<T>(const PartK<T> &, const SysK &, const CenK *, T *, T *, T *,  \
                                                 T *, cudaStream_t);                                           \
    template cudaError_t pm_launch_cic_umax<T>(const PartK<T> &, const T *, const T *, const T *, unsigned *,  \
                                               cudaStream_t);
