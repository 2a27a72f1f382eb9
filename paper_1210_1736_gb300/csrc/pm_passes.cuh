// FFT passes of the doubled-grid convolution (Sec. 2.1) on pair-packed mass
// sets: two real densities of one geometry (grids 2 and 3, or 4 and 5) travel
// as one complex field rho_a + i rho_b, so every transform is a plain complex
// FFT of power-of-two length and, H being real, the result is
// Phi_a + i Phi_b.  A set without partner uses rho_b = 0.
//
// Work array per pair: complex [z < nz][y < 2ny][kx < 2nx].
//   x forward : rows (z, y < ny), inputs x < nx (zero padding implicit)
//   y forward : columns (z, kx), inputs y < ny, all 2ny outputs
//   z convolve: columns (ky, kx), forward z (inputs z < nz), times the real,
//               even H-hat, inverse z, outputs z < nz
//   y inverse : columns (z, kx), all 2ny inputs, outputs y < ny
//   x inverse : rows (z, y < ny), outputs x < nx: Phi_b = Im, Phi_a + Phi_b
//
// Grid 1 (the fine grid, a set without partner) is solved for its
// difference fields: its z pass writes H-hat (D_x + i D_y) rho-hat to a
// second work array and H-hat (D_z + i) rho-hat in place, and its inverse
// passes run on both (fx + i fy, fz + i Phi_1).
//
// The column passes are persistent: each block walks tiles of COLS adjacent
// columns; a TMA tensor copy brings the next-but-one tile's input rows into
// shared memory (two buffers, mbarrier completion; the FP32 512-point y
// inverse keeps one and loads the next tile) while the block transforms the
// current one; every column pass stages its outputs in shared memory and
// sends them by TMA store.
#pragma once

#include <cuda.h>

#include "pm_fft.cuh"
#include "pm_launch.h"

namespace pmk {

// Programmatic dependent launch between the passes of a chain (they are
// launched with programmatic stream serialisation): a pass runs its
// prologue (twiddle tables, barriers), then waits until the previous pass
// has completed and its writes are visible before it touches the work
// array; each block signals, when it starts its last tile, that the next
// pass may be scheduled.  Both are no-ops for a plain launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

using pmfft::E;
using pmfft::nstages;
using pmfft::radix;

constexpr int NT = 256;  // threads per block of the x passes

template <int L> struct XShape {          // x passes: rows per block, padded row length
    static constexpr int TPC = L / E, LINES = NT / TPC, LDR = L + L / 16;
};

template <typename T, int L> constexpr size_t xpass_smem() {
    return (size_t)(pmfft::tw_total(L) + XShape<L>::LINES * XShape<L>::LDR) * sizeof(typename cplx_t<T>::type);
}


// ---------------------------------------------------------------------------
// x passes: the TPC = L/16 threads of a row are consecutive lanes, so a
// stage's inputs (rows t + k L/R) and the natural-order outputs are read and
// written straight between global memory and registers with warp-contiguous
// addresses; shared memory only carries the exchanges between stages, in a
// padded row private to the row's warp.
// ---------------------------------------------------------------------------
// x forward: z[x] = rho_a + i rho_b (scaled to mass), forward FFT of length
// L = 2nx, all L outputs written to the row of the work array.  Persistent:
// each block walks groups of LINES rows (the twiddle tables are built once).
template <typename T, int L>
__global__ void __launch_bounds__(NT) k_xfwd(const __grid_constant__ PassBatch B) {
    typedef typename cplx_t<T>::type C;
    typedef XShape<L> S;
    constexpr int NX = L / 2, NS = nstages(L);
    extern __shared__ __align__(16) unsigned char smraw[];
    C *tw = reinterpret_cast<C *>(smraw);
    C *sm = tw + pmfft::tw_total(L);
    const int tid = threadIdx.x, line = tid / S::TPC, t = tid % S::TPC;
    // the shape, twiddles and scale are the items' common ones; every field
    // is read into a register once (the stores below could otherwise make
    // the compiler reload them)
    const int ny = B.a[0].ny, lgi = B.lgi;
    // the items' arrays, copied once into shared memory (a parameter array
    // indexed at run time is read through slow generic loads)
    __shared__ const void *ip[PM_BATCH][3];
    if (tid < B.n) {
        ip[tid][0] = B.a[tid].rho_a;
        ip[tid][1] = B.a[tid].rho_b;
        ip[tid][2] = B.a[tid].work;
    }
    pmfft::expand_twiddles<L>(tw, static_cast<const C *>(B.a[0].tw));
    __syncthreads();
    pdl_wait();
    const long long nrows = (long long)ny * B.a[0].nz;
    const long long ngroups = (long long)B.n << lgi;   // row groups of every item
    const int lny = __ffs(ny) - 1;   // row r = z*ny + y; ny is a power of two
    const T scale = (T)B.a[0].scale;
    for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        if (grp + gridDim.x >= ngroups) pdl_release();
        const int item = (int)(grp >> lgi);
        const long long *rho_a = static_cast<const long long *>(ip[item][0]);
        const long long *rho_b = static_cast<const long long *>(ip[item][1]);
        C *work = static_cast<C *>(const_cast<void *>(ip[item][2]));
        const long long r = (grp & ((1LL << lgi) - 1)) * S::LINES + line;
        const bool valid = r < nrows;
        const long long *ra = rho_a + (valid ? r * NX : 0);
        const long long *rb = rho_b ? rho_b + (valid ? r * NX : 0) : nullptr;
        C v[E];
        constexpr int R0 = radix(L, 0, false);
#pragma unroll
        for (int kk = 0; kk < E / R0; ++kk)
#pragma unroll
            for (int q = 0; q < R0; ++q) {
                C val = czero<C>();
                if (valid && q < R0 / 2) {   // inputs x >= nx are the zero padding
                    const int x = pmfft::in_row<L, 0, false>(t, kk, q);
                    val.x = (T)__ldg(ra + x) * scale;
                    if (rb) val.y = (T)__ldg(rb + x) * scale;
                }
                v[kk * R0 + q] = val;
            }
        // a row's TPC threads are consecutive lanes of one warp and its
        // exchange row is private: the exchanges synchronise the warp only
        pmfft::fft_core<L, false, -1, true, false, true>(v, sm, pmfft::RowLayout{line * S::LDR}, t, tw);
        if (valid) {
            const long long z = r >> lny, y = r & (ny - 1);
            C *out = work + ((size_t)z * 2 * ny + y) * L;
            constexpr int RL = radix(L, NS - 1, false);
#pragma unroll
            for (int kk = 0; kk < E / RL; ++kk)
#pragma unroll
                for (int q = 0; q < RL; ++q) __stcg(out + pmfft::in_row<L, NS - 1, false>(t, kk, q), v[kk * RL + q]);
        }
    }
}

// x inverse: inverse FFT of length L = 2nx of each row y < ny; x < nx kept:
// Phi_b = Im, Phi_sum = Re + Im (or Re without partner; with a.split,
// Phi_sum = Re and Phi_b = Im).  Persistent as k_xfwd.
template <typename T, int L>
__global__ void __launch_bounds__(NT) k_xinv(const __grid_constant__ PassBatch B) {
    typedef typename cplx_t<T>::type C;
    typedef XShape<L> S;
    constexpr int NX = L / 2, NS = nstages(L);
    extern __shared__ __align__(16) unsigned char smraw[];
    C *tw = reinterpret_cast<C *>(smraw);
    C *sm = tw + pmfft::tw_total(L);
    const int tid = threadIdx.x, line = tid / S::TPC, t = tid % S::TPC;
    const int ny = B.a[0].ny, lgi = B.lgi;   // common to the items; read once (see k_xfwd)
    __shared__ void *ip[PM_BATCH][3];
    __shared__ int isplit[PM_BATCH];
    if (tid < B.n) {
        ip[tid][0] = B.a[tid].phi_b;
        ip[tid][1] = B.a[tid].phi_sum;
        ip[tid][2] = B.a[tid].work;
        isplit[tid] = B.a[tid].split;
    }
    pmfft::expand_twiddles<L>(tw, static_cast<const C *>(B.a[0].tw));
    __syncthreads();
    pdl_wait();
    const long long nrows = (long long)ny * B.a[0].nz;
    const long long ngroups = (long long)B.n << lgi;
    const int lny = __ffs(ny) - 1;   // row r = z*ny + y; ny is a power of two
    for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        if (grp + gridDim.x >= ngroups) pdl_release();
        const int item = (int)(grp >> lgi);
        T *phi_b = static_cast<T *>(ip[item][0]);
        T *phi_sum = static_cast<T *>(ip[item][1]);
        const bool split = isplit[item] != 0;
        const C *work = static_cast<const C *>(ip[item][2]);
        const long long r = (grp & ((1LL << lgi) - 1)) * S::LINES + line;
        const bool valid = r < nrows;
        const long long z = valid ? r >> lny : 0, y = valid ? r & (ny - 1) : 0;
        const C *in = work + ((size_t)z * 2 * ny + y) * L;
        C v[E];
        // the reversed plan, or the forward one where it closes with radix 2
        // (its exchange into that stage goes by shuffles)
        constexpr bool IREV = !pmfft::inv_fwd_plan(L);
        constexpr int R0 = radix(L, 0, IREV);
#pragma unroll
        for (int kk = 0; kk < E / R0; ++kk)
#pragma unroll
            for (int q = 0; q < R0; ++q)
                v[kk * R0 + q] = valid ? __ldg(in + pmfft::in_row<L, 0, IREV>(t, kk, q)) : czero<C>();
        pmfft::fft_core<L, IREV, 1, false, true, true>(v, sm, pmfft::RowLayout{line * S::LDR}, t, tw);
        if (valid) {
            T *phi_s = phi_sum + r * NX;
            constexpr int RL = radix(L, NS - 1, IREV);
#pragma unroll
            for (int kk = 0; kk < E / RL; ++kk)
#pragma unroll
                for (int q = 0; q < RL / 2; ++q) {   // outputs x < nx: registers q < RL/2 of the last stage
                    const int x = pmfft::in_row<L, NS - 1, IREV>(t, kk, q);
                    const C val = v[kk * RL + q];
                    // the arrays are global memory (pointers read from shared memory: say so)
                    if (split) {
                        __stcg(phi_s + x, val.x);
                        __stcg(phi_b + r * NX + x, val.y);
                    } else if (phi_b) {
                        __stcg(phi_b + r * NX + x, val.y);
                        __stcg(phi_s + x, val.x + val.y);
                    } else {
                        __stcg(phi_s + x, val.x);
                    }
                }
        }
    }
}

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase with a time limit (2 s); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, phase))
        if (globaltimer_ns() - t0 > 2000000000ull) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_addr(src))
                 : "memory");
}
// Plain bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing on an mbarrier.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until the committed stores have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until the committed stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Columns per tile and threads per block of the column passes (shared with
// the host, which encodes the tensor-map boxes).
template <typename T, int L> struct CShape {
    static constexpr int TPC = L / E;
    static constexpr int COLS = pm_col_cols(L, (int)sizeof(T));
    static constexpr int THREADS = COLS * TPC;
    static constexpr int EPC = sizeof(typename cplx_t<T>::type) / 8;   // 8-byte tensor elements per complex
};

template <int MODE> struct ColRows;       // input rows per tile for a transform of length L
template <> struct ColRows<COL_YFWD> { __host__ __device__ static constexpr int of(int L) { return L / 2; } };
template <> struct ColRows<COL_ZCONV> { __host__ __device__ static constexpr int of(int L) { return L / 2; } };
template <> struct ColRows<COL_YINV> { __host__ __device__ static constexpr int of(int L) { return L; } };

// Input buffers of the y pass: two (a tile prefetched two ahead), or one
// for the FP32 512-point inverse, whose 32 KB tiles would otherwise hold it
// to two blocks per SM by shared memory (one buffer: three, as its registers
// allow; the next tile's load still runs during this tile's transform, which
// has read its inputs into registers first).
template <typename T, int L, int MODE> __host__ __device__ constexpr int col_nbuf() {
    return (MODE == COL_YINV && L == 512 && sizeof(T) == 4) ? 1 : 2;
}
// Shared memory of a y pass: the input buffers, the exchange buffer and the
// stage twiddles of the one plan the pass runs (forward, or reversed for the
// inverse).
template <typename T, int L, int MODE> constexpr size_t col_smem() {
    typedef typename cplx_t<T>::type C;
    constexpr int COLS = CShape<T, L>::COLS;
    return 128 + (size_t)pmfft::tw_dir_size(L, MODE == COL_YINV) * sizeof(C) + (size_t)L * COLS * sizeof(C) +
           col_nbuf<T, L, MODE>() * (size_t)ColRows<MODE>::of(L) * COLS * sizeof(C) + 3 * 128;
}

// Persistent y pass (forward or inverse) over a batch: the items' maps
// B.lmap are 2D tensor maps over 8-byte elements whose box is
// (COLS * EPC, min(rows, 256)); an item's tile covers COLS columns of one z
// plane.  The outputs are staged in the exchange buffer, laid out [row][COLS]
// as a tile, and leave by tensor stores through B.smap (boxes of the output
// rows: 2ny for the forward, ny for the inverse; columns beyond nx2 are
// clipped by the copy).
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(CShape<T, L>::THREADS, 3) k_col(const __grid_constant__ PassBatch B) {
    typedef typename cplx_t<T>::type C;
    typedef CShape<T, L> S;
    constexpr int COLS = S::COLS, NS = nstages(L), ROWS = ColRows<MODE>::of(L);
    constexpr int BOXR = ROWS < 256 ? ROWS : 256, NBOX = ROWS / BOXR;
    constexpr unsigned TILE_BYTES = (unsigned)(ROWS * COLS * sizeof(C));
    constexpr bool REV_IN = (MODE == COL_YINV);
    constexpr int SIGN_IN = (MODE == COL_YINV) ? 1 : -1;
    constexpr int NBUF = col_nbuf<T, L, MODE>();

    extern __shared__ __align__(128) unsigned char smraw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smraw + 127) & ~(uintptr_t)127);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base);                 // 2 mbarriers
    C *buf0 = reinterpret_cast<C *>(base + 128);
    C *buf1 = NBUF == 2 ? buf0 + ROWS * COLS : buf0;
    C *sm = buf0 + NBUF * ROWS * COLS;
    // only this pass's plan's tables follow the exchange buffer: for the
    // reversed plan, the forward tables' offsets fall on the exchange
    // buffer's tail and are never read
    C *tw = sm + L * COLS - (REV_IN ? pmfft::tw_dir_size(L, false) : 0);
    const int tid = threadIdx.x;
    const int c = tid % COLS, t = tid / COLS;
    const int nx2 = 2 * B.a[0].nx, ny2 = 2 * B.a[0].ny;   // the items' common shape, read once
    int *const err = B.a[0].err;
    const long long tiles_per_z = (nx2 + COLS - 1) / COLS;   // a power of two, as nx2 and COLS
    const int ltpz = __ffs((int)tiles_per_z) - 1;
    const long long ntiles = (long long)B.n << B.lgi;
    const long long lmask = (1LL << B.lgi) - 1;

    // an item's tile -> TMA coordinates and the first column it covers
    auto coords = [&](long long lt, int &x, int &y) {
        x = (int)((lt & (tiles_per_z - 1)) * COLS * S::EPC);
        y = (int)((lt >> ltpz) * ny2);
    };
    auto issue = [&](long long tile, int b) {
        int x, y;
        coords(tile & lmask, x, y);
        const CUtensorMap *map = &B.lmap[tile >> B.lgi];
        C *dst = b ? buf1 : buf0;
        mbar_expect_tx(&bar[b], TILE_BYTES);
#pragma unroll
        for (int k = 0; k < NBOX; ++k) tma_load_2d(dst + k * BOXR * COLS, map, x, y + k * BOXR, &bar[b]);
    };

    __shared__ C *iwork[PM_BATCH];   // the items' work arrays (read once; see k_xfwd)
    if (tid < B.n) iwork[tid] = static_cast<C *>(B.a[tid].work);
    if (tid == 0) {
        for (int i = 0; i < B.n; ++i)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&B.lmap[i])) : "memory");
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    pmfft::expand_stage_twiddles<L, 1, REV_IN>(tw, static_cast<const C *>(B.a[0].tw));
    pmfft::expand_stage_twiddles<L, 2, REV_IN>(tw, static_cast<const C *>(B.a[0].tw));
    __syncthreads();
    pdl_wait();
    int issued[2] = {0, 0};   // loads issued per buffer (thread 0's count)
    if (tid == 0) {
        if (blockIdx.x < ntiles) { issue(blockIdx.x, 0); ++issued[0]; }
        if (NBUF == 2 && blockIdx.x + gridDim.x < ntiles) { issue(blockIdx.x + gridDim.x, 1); ++issued[1]; }
    }

    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        if (tile + gridDim.x >= ntiles) pdl_release();
        const int b = NBUF == 2 ? (it & 1) : 0;
        const unsigned phase = NBUF == 2 ? (unsigned)((it >> 1) & 1) : (unsigned)(it & 1);
        // a tensor copy that never lands: report, wait (bounded) for the other
        // copy in flight, stop; the decision is the same for the whole block
        if (!__syncthreads_and(mbar_wait(&bar[b], phase) ? 1 : 0)) {
            if (tid == 0) {
                atomicExch(err, 1);
                if (NBUF == 2) {
                    const int o = b ^ 1, used_o = it >> 1;   // uses of buffer o completed so far
                    if (issued[o] > used_o) mbar_wait(&bar[o], (unsigned)(used_o & 1));
                }
            }
            break;
        }
        const C *in = b ? buf1 : buf0;
        C v[E];
        constexpr int R0 = radix(L, 0, REV_IN);
        constexpr int OROWS = (MODE == COL_YFWD) ? L : L / 2, OBOX = OROWS < 256 ? OROWS : 256;
#pragma unroll
        for (int kk = 0; kk < E / R0; ++kk)
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const bool need = (MODE == COL_YINV) || r < R0 / 2;   // forward inputs above L/2 are padding
                v[kk * R0 + r] = need ? in[pmfft::in_row<L, 0, REV_IN>(t, kk, r) * COLS + c] : czero<C>();
            }
        // the previous tile's outputs have been read out of the exchange
        // buffer before this tile's stages write to it
        if (tid == 0) bulk_wait_read();
        __syncthreads();   // buffer b consumed, previous tile's exchange done
        if (tid == 0 && tile + NBUF * (long long)gridDim.x < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tile + NBUF * (long long)gridDim.x, b);
            ++issued[b];
        }

        static_assert(MODE == COL_YFWD || MODE == COL_YINV, "the z pass is k_colw");
        if constexpr (COLS * sizeof(C) == 64)   // FP32, L = 512: rows of 8 columns
            pmfft::fft_core<L, REV_IN, SIGN_IN, MODE != COL_YINV, MODE == COL_YINV, false>(
                v, sm, pmfft::ColLayoutHalf{COLS, c}, t, tw);
        else
            pmfft::fft_core<L, REV_IN, SIGN_IN, MODE != COL_YINV, MODE == COL_YINV>(v, sm, COLS, c, t, tw);
        // fft_core ends with a block barrier after its last exchange reads:
        // the exchange buffer takes the outputs, rows in_row of the last
        // stage (the inverse keeps rows < L/2: registers r < RL/2)
        {
            constexpr bool REV_OUT = (MODE == COL_YINV);
            constexpr int RL = radix(L, NS - 1, REV_OUT), RK = (MODE == COL_YFWD) ? RL : RL / 2;
#pragma unroll
            for (int kk = 0; kk < E / RL; ++kk)
#pragma unroll
                for (int r = 0; r < RK; ++r) sm[pmfft::in_row<L, NS - 1, REV_OUT>(t, kk, r) * COLS + c] = v[kk * RL + r];
        }
        fence_async_smem();   // the staged outputs are visible to the tensor copies
        __syncthreads();
        if (tid == 0) {
            int x, y;
            coords(tile & lmask, x, y);
            const CUtensorMap *smap = &B.smap[tile >> B.lgi];
#pragma unroll
            for (int k = 0; k < OROWS / OBOX; ++k) tma_store_2d(smap, x, y + k * OBOX, sm + k * OBOX * COLS);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();   // the stores have read the buffer before the block leaves
}


// ---------------------------------------------------------------------------
// z pass (forward z FFT, times H-hat, inverse z FFT) with warp-private
// transforms.  A tile is COLS adjacent (ky, kx) columns whose nz = L/2 input
// rows a TMA copy brings into a swizzled buffer of NSUB sub-tiles [rows][SW]
// (SW columns fill one 32/64/128-byte row; the tensor map's swizzle and this
// kernel's address function agree, so the first-stage reads are free of bank
// conflicts).  The L/16 threads of a column are consecutive lanes of one
// warp, so the stage exchanges use a private padded row per column and
// synchronise the warp only (and the exchange into a closing radix-2 stage,
// at L = 32 and 512, goes by shuffles).  For L = 128, 256 the tile's H-hat
// rows arrive by one bulk copy into the consumed input buffer during the
// forward FFT.
// The outputs (rows < L/2) are staged into the tile's own buffer and leave by
// TMA store; the buffer then takes the prefetch of the tile two steps ahead.
// (The same structure measured slower than k_col for the y passes, so those
// stay there.)
// ---------------------------------------------------------------------------
// Order of the z pass's H-hat table within one octant column (L values).
// Register order (entry e*TPC + t for register e of thread t) lets the TPC
// lanes of a column read consecutive values with each load; with TPC <= 4
// (L <= 64) one such load touches a sector per column and uses half of it,
// so short transforms take thread-major order (entries t*E .. t*E + E-1,
// read as 16-byte vectors).
__host__ __device__ constexpr bool hhat_thread_major(int L) { return L <= 64; }

template <typename T, int L> struct WShape {
    typedef typename cplx_t<T>::type C;
    static constexpr int TPC = L / E;
    static constexpr int COLS = pm_col_cols(L, (int)sizeof(T));
    static constexpr int THREADS = COLS * TPC;
    static constexpr int SW = pm_zsub_cols(L, (int)sizeof(T));
    static constexpr int NSUB = COLS / SW;
    static constexpr int P = SW * (int)sizeof(C);                 // bytes per sub-tile row
    static constexpr int RIN = L / 2;                             // input and output rows per column
    static constexpr int BOXI = RIN < 256 ? RIN : 256, NBOXI = RIN / BOXI;
    static constexpr int LDR = L + L / 16;
    static constexpr int EPC = (int)sizeof(C) / 8;
    static constexpr unsigned BUF = (unsigned)(RIN * COLS * sizeof(C));
    static constexpr int HS = pm_hhat_stride(L);                       // H-hat values per octant column
    static constexpr unsigned HBYTES = (unsigned)(COLS * HS * sizeof(T));   // a tile's staged H-hat rows
    static_assert(HBYTES <= BUF, "a tile's H-hat rows fit its input buffer");
    // the longest transform runs two blocks per SM with the warps decoupled
    // (thread 0 sends a tile once every warp has arrived on its barrier); the
    // others measured faster block-synchronous (block barriers per tile)
    static constexpr bool FREE = L >= 512;
};

// Shared memory of the z pass: two tile buffers, the exchange rows, the
// stage twiddles, six mbarriers, and (decoupled warps, L >= 512) one H-hat
// column per warp, prefetched with cp.async while the forward FFT runs.
template <typename T, int L> constexpr size_t colw_smem() {
    typedef WShape<T, L> S;
    return 1024 + 2 * (size_t)S::BUF + (size_t)S::COLS * S::LDR * sizeof(typename S::C) +
           (size_t)pmfft::tw_total(L) * sizeof(typename S::C) + 64 +
           (S::FREE ? (size_t)(S::THREADS / 32) * S::HS * sizeof(T) : 0);
}

// Asynchronous global -> shared copies of 16 bytes (both addresses 16-byte
// aligned), completed by cp_async_wait_all in the issuing thread.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Byte offset of element (row, column c) of a tile buffer whose sub-tiles
// hold ROWS rows (swizzle of the tensor map: the 16-byte chunk index XOR the
// index bits of the 128-byte line).
template <typename T, int L, int ROWS>
__device__ __forceinline__ uint32_t woff(int row, int c) {
    typedef WShape<T, L> S;
    const uint32_t o = (uint32_t)row * S::P + (uint32_t)(c % S::SW) * (uint32_t)sizeof(typename S::C);
    const uint32_t sw = S::P >= 32 ? (o ^ (((o >> 7) & (uint32_t)(S::P / 16 - 1)) << 4)) : o;
    return (uint32_t)(c / S::SW) * (uint32_t)(ROWS * S::P) + sw;
}

// Over a batch: B.lmap, the items' maps with boxes (SW*EPC, min(nz, 256)),
// for the loads; B.smap, the same boxes, for the stores (the same map in
// place, another work array's for the first difference-field pass).  DM = 0:
// the spectral factor is H-hat; DM = 1 (difference fields): H-hat
// (D_x + i D_y) for dmode 1, H-hat (D_z + i) for dmode 2 (see PairArgs);
// DM = 2 (dmode 3, L <= 256): both from one forward transform, the first
// products' outputs stored through smap, the second's in place through
// lmap.  The modes are separate instantiations so that the plain pass
// carries no mode branch.
template <typename T, int L, int DM>
__global__ void __launch_bounds__(WShape<T, L>::THREADS, ((L >= 512 || DM == 2) ? 2 : 3))
    k_colw(const __grid_constant__ PassBatch B) {
    typedef WShape<T, L> S;
    typedef typename S::C C;
    constexpr int NS = nstages(L), NWARPS = S::THREADS / 32;
    constexpr bool FREE = S::FREE;
    // the inverse runs the reversed plan (its first stage takes the forward's
    // last-stage registers as they are), or the forward plan where that
    // closes with radix 2 (registers renamed; the exchange into the radix-2
    // stage goes by shuffles)
    constexpr bool IREV = !pmfft::inv_fwd_plan(L);
    extern __shared__ __align__(128) unsigned char smraw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    C *xch = reinterpret_cast<C *>(base + 2 * S::BUF);
    C *tw = xch + S::COLS * S::LDR;
    uint64_t *full = reinterpret_cast<uint64_t *>(tw + pmfft::tw_total(L));   // tile loaded (tx bytes)
    uint64_t *staged = full + 2;                                            // every warp staged (FREE)
    uint64_t *hfull = staged + 2;                                           // tile's H-hat staged
    T *hpre = reinterpret_cast<T *>(hfull + 2);   // FREE: one prefetched H-hat column per warp (16-byte aligned)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = lane % S::TPC;
    const int c = warp * (32 / S::TPC) + lane / S::TPC;   // column within the tile
    const PairArgs &a = B.a[0];   // the shape, tables and mode are the items' common ones
    const int nx2 = 2 * a.nx, ny2 = 2 * a.ny, lnx2 = __ffs(nx2) - 1;
    // tile indices fit in 32 bits: at most 8 items of (2 * 256)^2 / COLS tiles
    const int lgi = B.lgi, lmask = (1 << lgi) - 1;

    // an item's tile <-> sub-tiles of the buffer, each NBOXI boxes of BOXI rows
    auto issue_load = [&](int tile, int b) {
        const CUtensorMap *map = &B.lmap[tile >> lgi];
        const int lt = tile & lmask;
        mbar_expect_tx(&full[b], S::BUF);
#pragma unroll
        for (int s = 0; s < S::NSUB; ++s)
#pragma unroll
            for (int k = 0; k < S::NBOXI; ++k)
                tma_load_2d(base + b * S::BUF + s * S::RIN * S::P + k * S::BOXI * S::P, map,
                            (int)((lt * S::COLS + s * S::SW) * S::EPC), k * S::BOXI, &full[b]);
    };
    auto issue_store = [&](int tile, const unsigned char *src, bool to_lmap = false) {
        const CUtensorMap *smap = to_lmap ? &B.lmap[tile >> lgi] : &B.smap[tile >> lgi];
        const int lt = tile & lmask;
#pragma unroll
        for (int s = 0; s < S::NSUB; ++s)
#pragma unroll
            for (int k = 0; k < S::NBOXI; ++k)
                tma_store_2d(smap, (int)((lt * S::COLS + s * S::SW) * S::EPC), k * S::BOXI,
                             src + s * S::RIN * S::P + k * S::BOXI * S::P);
    };

    __shared__ const T *ihhat[PM_BATCH];   // the items' H-hat tables (read once; see k_xfwd)
    if (tid < B.n) ihhat[tid] = static_cast<const T *>(B.a[tid].hhat);
    if (tid == 0) {
        for (int i = 0; i < B.n; ++i) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&B.lmap[i])) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&B.smap[i])) : "memory");
        }
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&staged[0], NWARPS);
        mbar_init(&staged[1], NWARPS);
        mbar_init(&hfull[0], 1);
        mbar_init(&hfull[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // H-hat staging: with block barriers and a tile inside one ky row (COLS
    // <= nx), the tile's H-hat rows (kyr fixed, kxr ascending for kx < nx,
    // descending from nx for kx >= nx) are one contiguous block of exactly
    // BUF bytes; it is copied into the tile's input buffer once the inputs
    // are in registers and read from there for the multiply
    const bool hstage = !FREE && L >= 128 && S::COLS <= a.nx;
    if (DM == 2 && !hstage && !hhat_thread_major(L)) {   // the fused mode's H-hat sources (the host checks)
        if (threadIdx.x == 0) atomicExch(a.err, 2);   // a launch the kernel does not support (not a wait)
        return;
    }
    bool hpend = false;   // thread 0: an H-hat copy not yet seen complete
    pmfft::expand_twiddles<L>(tw, static_cast<const C *>(a.tw));
    __syncthreads();
    pdl_wait();
    // thread 0 issues every copy; counts per buffer of loads issued and of
    // tiles sent (to drain after an expired wait)
    int issued0 = 0, issued1 = 0, done0 = 0, done1 = 0;
    const int nt0 = B.n << lgi;
    int deferred = -1;   // thread 0: tile whose buffer awaits its refill
    if (tid == 0) {
        if ((int)blockIdx.x < nt0) { issue_load(blockIdx.x, 0); ++issued0; }
        if ((int)(blockIdx.x + gridDim.x) < nt0) { issue_load(blockIdx.x + gridDim.x, 1); ++issued1; }
    }
    const pmfft::RowLayout lay{c * S::LDR};
    bool failed = false;

    int it = 0;
    const int nt = nt0;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x, ++it) {
        if (tile + (int)gridDim.x >= nt) pdl_release();
        const int b = it & 1;
        const unsigned phase = (unsigned)((it >> 1) & 1);
        if (FREE) {
            if (!mbar_wait(&full[b], phase)) { failed = true; break; }
        } else if (!__syncthreads_and(mbar_wait(&full[b], phase) ? 1 : 0)) {
            failed = true;
            break;
        }
        unsigned char *in = base + b * S::BUF;
        const int lt = tile & lmask;                       // the tile within its item
        const T *hhat = ihhat[tile >> lgi];
        if constexpr (FREE) {
            // this warp's column (one per warp): its H-hat column lands in
            // shared memory while the forward FFT runs
            const int qc = lt * S::COLS + c;
            const int ky = qc >> lnx2, kx = qc & (nx2 - 1);
            const int kyr = ky <= a.ny ? ky : ny2 - ky, kxr = kx <= a.nx ? kx : nx2 - kx;
            const unsigned char *src =
                reinterpret_cast<const unsigned char *>(hhat + ((size_t)kyr * (a.nx + 1) + kxr) * S::HS);
            unsigned char *dst = reinterpret_cast<unsigned char *>(hpre + warp * S::HS);
            for (int ch = lane; ch < (int)(S::HS * sizeof(T) / 16); ch += 32) cp_async16(dst + 16 * ch, src + 16 * ch);
            cp_async_commit();
        }
        C v[E];
        constexpr int R0 = radix(L, 0, false);
#pragma unroll
        for (int kk = 0; kk < E / R0; ++kk)
#pragma unroll
            for (int r = 0; r < R0; ++r)
                v[kk * R0 + r] = (r < R0 / 2)   // inputs above nz are the padding
                                     ? *reinterpret_cast<const C *>(
                                           in + woff<T, L, S::RIN>(pmfft::in_row<L, 0, false>(t, kk, r), c))
                                     : czero<C>();
        // A column's elements are touched only by the lanes of that column,
        // and the exchanges synchronise the warp, so the outputs may
        // overwrite this buffer without a block barrier; the block-synchronous
        // variant keeps the warps in step.
        if (!FREE) __syncthreads();
        if (!FREE && tid == 0 && deferred >= 0) {
            // the previous tile's store has long read its buffer by now: the
            // wait is short, and the refill (the tile after this one) still
            // lands well before it is needed
            bulk_wait_read();
            const int db = b ^ 1;
            if (deferred + 2 * (int)gridDim.x < nt) {
                issue_load(deferred + 2 * (int)gridDim.x, db);
                if (db) ++issued1; else ++issued0;
            }
            deferred = -1;
        }
        const int q0 = lt * S::COLS;
        const int k0 = (int)(q0 & (nx2 - 1));
        if (hstage && tid == 0) {
            const int ky0 = (int)(q0 >> lnx2);
            const int kyr0 = ky0 <= a.ny ? ky0 : ny2 - ky0;
            const int r0 = k0 < a.nx ? k0 : nx2 - k0 - S::COLS + 1;
            fence_async_smem();   // the inputs' generic reads before the copy's writes
            mbar_expect_tx(&hfull[b], S::HBYTES);
            bulk_load(in, hhat + ((size_t)kyr0 * (a.nx + 1) + r0) * S::HS, S::HBYTES, &hfull[b]);
            hpend = true;
        }

        pmfft::fft_core<L, false, -1, true, false, true>(v, xch, lay, t, tw);
        // spectral factor of this column: H-hat times 1, D_x + i D_y
        // (column constant) or D_z + i (per register: kz of register e is
        // the last forward stage's output row)
        C dxy = czero<C>();
        if ((DM == 1 && a.dmode == 1) || DM == 2) {
            const int qc = lt * S::COLS + c;
            const C ex = static_cast<const C *>(a.dtx)[qc & (nx2 - 1)];
            const C ey = static_cast<const C *>(a.dty)[qc >> lnx2];
            dxy.x = ex.x - ey.y;
            dxy.y = ex.y + ey.x;
        }
        // mirrored kz (0..L/2) of register e: the last forward stage's row
        auto kz_mirror = [&](int e) {
            constexpr int RLF = radix(L, NS - 1, false);
            const int kz = pmfft::in_row<L, NS - 1, false>(t, e / RLF, e % RLF);
            return kz <= L / 2 ? kz : L - kz;
        };
        auto hmul = [&](int e, T h) {
            if constexpr (DM == 0) {
                v[e].x *= h;
                v[e].y *= h;
                return;
            }
            C f = dxy;
            if (a.dmode == 2) {
                constexpr int RLF = radix(L, NS - 1, false);
                const int kz = pmfft::in_row<L, NS - 1, false>(t, e / RLF, e % RLF);
                f = static_cast<const C *>(a.dtz)[kz];
                f.y += (T)1;
            }
            f.x *= h;
            f.y *= h;
            v[e] = cmul(v[e], f);
        };
        // DM == 2: both difference fields from the one forward transform:
        // u = S H-hat (D_x + i D_y) -> fx + i fy (work2, through smap), then
        // v = S H-hat (D_z + i) -> fz + i Phi_1 (in place, through lmap, by
        // the common code below).  hz: the column's H-hat values, indexed by
        // the mirrored kz (staged rows) or by the register (thread-major
        // table); false after an expired wait (the caller stops).
        auto fused = [&](const T *hz, bool mirrored, bool ok) -> bool {
            C u[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                constexpr int RLF = radix(L, NS - 1, false);
                const int kz = pmfft::in_row<L, NS - 1, false>(t, e / RLF, e % RLF);
                const T h = mirrored ? hz[kz <= L / 2 ? kz : L - kz] : __ldg(hz + e);
                C f1 = dxy, f2 = static_cast<const C *>(a.dtz)[kz];
                f2.y += (T)1;
                f1.x *= h; f1.y *= h;
                f2.x *= h; f2.y *= h;
                u[e] = cmul(v[e], f1);
                v[e] = cmul(v[e], f2);
            }
            if constexpr (!IREV) pmfft::regs_last_to_first<L>(u);
            pmfft::fft_core<L, IREV, 1, false, true, true>(u, xch, lay, t, tw);
            // every H-hat read done before the outputs overwrite the buffer
            if (!__syncthreads_and(ok ? 1 : 0)) {
                failed = true;
                if (tid == 0 && hpend) mbar_wait(&hfull[b], phase);   // let the copy land (bounded)
                return false;
            }
            {
                constexpr int RL = radix(L, NS - 1, IREV);
#pragma unroll
                for (int kk = 0; kk < E / RL; ++kk)
#pragma unroll
                    for (int r = 0; r < RL / 2; ++r)
                        *reinterpret_cast<C *>(in + woff<T, L, S::RIN>(pmfft::in_row<L, NS - 1, IREV>(t, kk, r), c)) =
                            u[kk * RL + r];
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                issue_store(tile, in);
                bulk_commit();
                bulk_wait_read();   // read out before the second outputs overwrite the buffer
            }
            __syncthreads();
            if constexpr (!IREV) pmfft::regs_last_to_first<L>(v);
            pmfft::fft_core<L, IREV, 1, false, true, true>(v, xch, lay, t, tw);
            return true;
        };
        bool hok = true;
        if (hstage) {
            // H-hat of column c from the staged rows (row c, or COLS-1-c
            // for the mirrored half), indexed by the register's mirrored kz
            hok = mbar_wait(&hfull[b], phase);
            if (hok && tid == 0) hpend = false;
            const T *hz = reinterpret_cast<const T *>(in) + (k0 < a.nx ? c : S::COLS - 1 - c) * S::HS;
            if constexpr (DM == 2) {
                if (!fused(hz, true, hok)) break;
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) hmul(e, hz[kz_mirror(e)]);
                if constexpr (!IREV) pmfft::regs_last_to_first<L>(v);
                pmfft::fft_core<L, IREV, 1, false, true, true>(v, xch, lay, t, tw);
                // every H-hat read done before the outputs overwrite the buffer
                if (!__syncthreads_and(hok ? 1 : 0)) {
                    failed = true;
                    if (tid == 0 && hpend) mbar_wait(&hfull[b], phase);   // let the copy land (bounded)
                    break;
                }
            }
        } else {
            // H-hat of column (kyr, kxr), stored by pm_store_hhat in the
            // order hhat_thread_major gives for L
            const int q = lt * S::COLS + c;
            const int ky = q >> lnx2, kx = q & (nx2 - 1);   // nx2 is a power of two
            const int kyr = ky <= a.ny ? ky : ny2 - ky;
            const int kxr = kx <= a.nx ? kx : nx2 - kx;
            const T *hcol = hhat + ((size_t)kyr * (a.nx + 1) + kxr) * S::HS;
            if constexpr (DM == 2 && hhat_thread_major(L)) {
                if (!fused(hcol + t * E, false, true)) break;
            } else if constexpr (hhat_thread_major(L)) {
                const T *hz = hcol + t * E;   // 16-byte aligned: L, E multiples of 16
                if constexpr (sizeof(T) == 4) {
#pragma unroll
                    for (int e = 0; e < E; e += 4) {
                        const float4 h = __ldg(reinterpret_cast<const float4 *>(hz + e));
                        hmul(e, h.x); hmul(e + 1, h.y); hmul(e + 2, h.z); hmul(e + 3, h.w);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < E; e += 2) {
                        const double2 h = __ldg(reinterpret_cast<const double2 *>(hz + e));
                        hmul(e, h.x); hmul(e + 1, h.y);
                    }
                }
            } else if constexpr (FREE) {
                cp_async_wait_all();
                __syncwarp();
                const T *hz = hpre + warp * S::HS;
#pragma unroll
                for (int e = 0; e < E; ++e) hmul(e, hz[kz_mirror(e)]);
                __syncwarp();   // every lane's reads done before the next tile's prefetch
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) hmul(e, __ldg(hcol + kz_mirror(e)));
            }
            if constexpr (DM != 2) {   // (the fused mode ran both inverses)
                if constexpr (!IREV) pmfft::regs_last_to_first<L>(v);
                pmfft::fft_core<L, IREV, 1, false, true, true>(v, xch, lay, t, tw);
            }
        }
        {
            // inverse outputs below L/2: registers r < RL/2 of the last
            // stage of the inverse's plan
            constexpr int RL = radix(L, NS - 1, IREV);
#pragma unroll
            for (int kk = 0; kk < E / RL; ++kk)
#pragma unroll
                for (int r = 0; r < RL / 2; ++r)
                    *reinterpret_cast<C *>(in + woff<T, L, S::RIN>(pmfft::in_row<L, NS - 1, IREV>(t, kk, r), c)) =
                        v[kk * RL + r];
        }
        fence_async_smem();   // the staged outputs are visible to the tensor copies
        if (FREE) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&staged[b]);
        } else {
            __syncthreads();
        }
        if (tid == 0) {
            if (FREE && !mbar_wait(&staged[b], phase)) { failed = true; break; }
            issue_store(tile, in, DM == 2);   // the fused pass's second outputs go back in place
            bulk_commit();
            if (b) ++done1; else ++done0;
            if (FREE) {
                bulk_wait_read();   // the staged outputs have been read out
                if (tile + 2 * (int)gridDim.x < nt) {
                    issue_load(tile + 2 * (int)gridDim.x, b);
                    if (b) ++issued1; else ++issued0;
                }
            } else {
                deferred = tile;    // buffer b is refilled once the store has read it
            }
        }
    }
    if (failed) atomicExch(a.err, 1);
    if (tid == 0) {
        bulk_wait_all();
        // loads still in flight after an expired wait land before the block
        // leaves (bounded)
        if (issued0 > done0) mbar_wait(&full[0], (unsigned)(done0 & 1));
        if (issued1 > done1) mbar_wait(&full[1], (unsigned)(done1 & 1));
    }
}

}  // namespace pmk
