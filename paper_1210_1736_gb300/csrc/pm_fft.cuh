// Register/shared-memory FFT building blocks for the doubled-grid convolution
// (Sec. 2.1: the potential of the isolated system from the 2N-periodic
// convolution, evaluated with FFTs of length L = 2N per axis).
//
// Each transform of length L is done by L/16 threads holding 16 values each;
// stages are radix-16 (plus one radix-2/4/8 stage where L is not a power of
// 16) in the self-sorting Stockham order, exchanging through shared memory
// laid out so that a warp's accesses are conflict-free, or, into a closing
// radix-2 stage of a transform held by one warp, by warp shuffles.
#pragma once

#include "pm_internal.cuh"

namespace pmfft {

constexpr int E = 16;  // values held per thread

__host__ __device__ constexpr int nstages(int L) { return L <= 16 ? 1 : (L <= 256 ? 2 : 3); }
// Forward plan: 16 | 16,L/16 | 16,16,2 (L = 512).
__host__ __device__ constexpr int fwd_radix(int L, int s) {
    return s == 0 ? 16 : (L == 512 ? (s == 1 ? 16 : 2) : L / 16);
}
// A plan is the forward plan or its reverse; reversing lets the first stage
// of an inverse transform take the forward transform's last-stage registers
// as they are (see also inv_fwd_plan).
__host__ __device__ constexpr int radix(int L, int s, bool rev) {
    return rev ? fwd_radix(L, nstages(L) - 1 - s) : fwd_radix(L, s);
}
__host__ __device__ constexpr int stride_before(int L, int s, bool rev) {
    return s == 0 ? 1 : stride_before(L, s - 1, rev) * radix(L, s - 1, rev);
}

// Per-stage twiddle tables, laid out so that register r of a thread with
// j % Ns = jm reads entry r*Ns + jm (consecutive jm: consecutive addresses):
// table of stage S (S > 0) = w^{(jm r L / (Ns R)) mod L}, r < R, jm < Ns, with
// w = exp(-2 pi i / L).  The forward plan's tables come first, then the
// reversed plan's.
__host__ __device__ constexpr int tw_stage_size(int L, int S, bool rev) {
    return S == 0 ? 0 : stride_before(L, S, rev) * radix(L, S, rev);
}
__host__ __device__ constexpr int tw_dir_size(int L, bool rev) {
    return tw_stage_size(L, 1, rev) * (nstages(L) > 1) + tw_stage_size(L, 2, rev) * (nstages(L) > 2);
}
__host__ __device__ constexpr int tw_offset(int L, int S, bool rev) {
    return (rev ? tw_dir_size(L, false) : 0) + (S >= 2 ? tw_stage_size(L, 1, rev) : 0);
}
__host__ __device__ constexpr int tw_total(int L) { return tw_dir_size(L, false) + tw_dir_size(L, true); }

template <int L, int S, bool REV, typename C>
__device__ __forceinline__ void expand_stage_twiddles(C *tab, const C *g) {
    if (S >= nstages(L)) return;
    constexpr int Ns = stride_before(L, S, REV), R = radix(L, S, REV), OFF = tw_offset(L, S, REV);
    for (int i = threadIdx.x; i < Ns * R; i += blockDim.x) {
        const int r = i / Ns, jm = i % Ns;
        tab[OFF + i] = g[(jm * r * (L / (Ns * R))) & (L - 1)];
    }
}
// Builds the stage tables in shared memory from the plain table
// g[m] = w^m, m < L (the caller synchronises before use).
template <int L, typename C> __device__ __forceinline__ void expand_twiddles(C *tab, const C *g) {
    expand_stage_twiddles<L, 1, false>(tab, g);
    expand_stage_twiddles<L, 2, false>(tab, g);
    expand_stage_twiddles<L, 1, true>(tab, g);
    expand_stage_twiddles<L, 2, true>(tab, g);
}

// z * exp(SIGN * 2 pi i e / 16) for a compile-time-known e.
template <int SIGN, typename C> __device__ __forceinline__ C rot16(int e, C z) {
    typedef decltype(z.x) T;
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173,
            r2 = (T)0.70710678118654752440;
    e &= 15;
    T c = 0, s = 0;
    switch (e) {
        case 0: return z;
        case 4: return cmul_i<SIGN>(z);
        case 8: { C r; r.x = -z.x; r.y = -z.y; return r; }
        case 12: return cmul_i<-SIGN>(z);
        case 1: c = c1; s = s1; break;
        case 2: c = r2; s = r2; break;
        case 3: c = s1; s = c1; break;
        case 5: c = -s1; s = c1; break;
        case 6: c = -r2; s = r2; break;
        case 7: c = -c1; s = s1; break;
        case 9: c = -c1; s = -s1; break;
        case 10: c = -r2; s = -r2; break;
        case 11: c = -s1; s = -c1; break;
        case 13: c = s1; s = -c1; break;
        case 14: c = r2; s = -r2; break;
        case 15: c = c1; s = -s1; break;
    }
    if (SIGN < 0) s = -s;
    C r;
    r.x = z.x * c - z.y * s;
    r.y = z.x * s + z.y * c;
    return r;
}

// In-register DFT of length R (natural order in and out):
// X[k] = sum_r v[r] exp(SIGN 2 pi i r k / R).
template <int R, int SIGN, typename C> struct Dft;

template <int SIGN, typename C> struct Dft<1, SIGN, C> {
    static __device__ __forceinline__ void run(C *) {}
};
template <int SIGN, typename C> struct Dft<2, SIGN, C> {
    static __device__ __forceinline__ void run(C *v) {
        C a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
        v[0] = a; v[1] = b;
    }
};
template <int SIGN, typename C> struct Dft<4, SIGN, C> {
    static __device__ __forceinline__ void run(C *v) {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = cmul_i<SIGN>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
    }
};
// Cooley-Tukey split R = N1*N2: input n = N2*n1 + n2, output k = k1 + N1*k2.
template <int N1, int N2, int SIGN, typename C>
__device__ __forceinline__ void dft_split(C *v) {
    C y[N1 * N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
        C t[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) t[n1] = v[N2 * n1 + n2];
        Dft<N1, SIGN, C>::run(t);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) y[n2 * N1 + k1] = rot16<SIGN>((16 / (N1 * N2)) * n2 * k1, t[k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        C t[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) t[n2] = y[n2 * N1 + k1];
        Dft<N2, SIGN, C>::run(t);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k1 + N1 * k2] = t[k2];
    }
}
template <int SIGN, typename C> struct Dft<8, SIGN, C> {
    static __device__ __forceinline__ void run(C *v) { dft_split<2, 4, SIGN>(v); }
};
template <int SIGN, typename C> struct Dft<16, SIGN, C> {
    static __device__ __forceinline__ void run(C *v) { dft_split<4, 4, SIGN>(v); }
};

// Radix 16 as 4 x 4 with two prunings of the doubled-grid transforms:
// ZIN: inputs 8..15 are zero (the padding half of a forward input), so each
// first-level DFT4 has two nonzero inputs; HOUT: only outputs 0..7 are kept
// (the active half of an inverse output), so each final DFT4 computes two.
template <int SIGN, bool ZIN, bool HOUT, typename C>
__device__ __forceinline__ void dft16(C *v) {
    C y[16];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C t[4];
        if (ZIN) {
            const C a = v[n2], b = v[4 + n2], wb = cmul_i<SIGN>(b);
            t[0] = cadd(a, b); t[1] = cadd(a, wb); t[2] = csub(a, b); t[3] = csub(a, wb);
        } else {
            t[0] = v[n2]; t[1] = v[4 + n2]; t[2] = v[8 + n2]; t[3] = v[12 + n2];
            Dft<4, SIGN, C>::run(t);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2 * 4 + k1] = rot16<SIGN>(n2 * k1, t[k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        const C t0 = y[k1], t1 = y[4 + k1], t2 = y[8 + k1], t3 = y[12 + k1];
        if (HOUT) {
            v[k1] = cadd(cadd(t0, t2), cadd(t1, t3));
            v[k1 + 4] = cadd(csub(t0, t2), cmul_i<SIGN>(csub(t1, t3)));
        } else {
            C t[4] = {t0, t1, t2, t3};
            Dft<4, SIGN, C>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
        }
    }
}

// Butterflies of stage S on the thread's E registers.  Thread t of a column
// owns the stage items j = t + kk*TPC (kk < E/R); register kk*R + r holds the
// input x[j + r*L/R] and afterwards the output y[(j/Ns)*Ns*R + j%Ns + r*Ns].
// tw: the stage tables of expand_twiddles (conjugated for SIGN > 0).
// ZIN / HOUT select the pruned radix-16 (see dft16); they are only passed
// for radix-16 stages.
template <int L, int S, bool REV, int SIGN, bool ZIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void stage_butterflies(C *v, int t, const C *tw) {
    constexpr int R = radix(L, S, REV), Ns = stride_before(L, S, REV), TPC = L / E;
    if constexpr (R == 2 && Ns == L / 2) {
        // a closing radix-2 stage: item j = t + kk TPC has the twiddle
        // w^j = w^t exp(-2 pi i kk / 16) (w^TPC = exp(-2 pi i / 16)): one
        // table entry per thread, the rest constant rotations.  HOUT keeps
        // the output rows < L/2 only (register kk*2).
        const C wt = tw[tw_offset(L, S, REV) + Ns + t];
#pragma unroll
        for (int kk = 0; kk < E / 2; ++kk) {
            const C b = rot16<SIGN>(kk, (SIGN < 0) ? cmul(v[2 * kk + 1], wt) : cconjmul(v[2 * kk + 1], wt));
            const C a = v[2 * kk];
            v[2 * kk] = cadd(a, b);
            if (!HOUT) v[2 * kk + 1] = csub(a, b);
        }
    } else {
#pragma unroll
        for (int kk = 0; kk < E / R; ++kk) {
            const int j = t + kk * TPC;
            if (Ns > 1) {
                const C *tws = tw + tw_offset(L, S, REV) + (j % Ns);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = tws[r * Ns];
                    v[kk * R + r] = (SIGN < 0) ? cmul(v[kk * R + r], w) : cconjmul(v[kk * R + r], w);
                }
            }
            if (R == 16 && (ZIN || HOUT)) dft16<SIGN, ZIN, HOUT>(v + kk * R);
            else Dft<R, SIGN, C>::run(v + kk * R);
        }
    }
}

// Row of the output of register (kk, r) of stage S.
template <int L, int S, bool REV>
__device__ __forceinline__ int out_row(int t, int kk, int r) {
    constexpr int R = radix(L, S, REV), Ns = stride_before(L, S, REV), TPC = L / E;
    const int j = t + kk * TPC;
    return (j / Ns) * Ns * R + (j % Ns) + r * Ns;
}
// Row of the input of register (kk, r) of stage S.
template <int L, int S, bool REV>
__device__ __forceinline__ int in_row(int t, int kk, int r) {
    constexpr int R = radix(L, S, REV), TPC = L / E;
    return t + kk * TPC + r * (L / R);
}

// Shared-memory layouts of the exchange between stages.  A layout maps the
// row (FFT index) of the calling thread's transform to an element offset.
struct ColLayout {              // [row][ldc] array, transform = column c
    int ldc, c;
    __device__ __forceinline__ int operator()(int row) const { return row * ldc + c; }
};
// [row][ldc] array of 64-byte rows (half the banks; 8-byte accesses run in
// half-warps, two rows of a column group at once).  Row `row` is stored at
// row ^ flip(row), flip = parity of row bits 1 and 4, so that the two rows a
// half-warp touches (1 apart from an even row, 2 apart in a radix-2 first
// stage, 16 apart in a radix-16 first stage) land on different bank halves;
// a bijection of [0, L).  Every exchange row of a stage is X | K, X from the
// thread and K a compile-time constant on disjoint bits, and flip is linear
// in the bits, so the offset is one of two per-thread bases plus a constant
// (store_stage / load_stage below): no address arithmetic per access.
struct ColLayoutHalf {
    int ldc, c;
    __host__ __device__ static constexpr int flip(int x) { return ((x >> 1) ^ (x >> 4)) & 1; }
    // offset of X | K = base(X, flip(K) ^ (K & 1)) + (K & ~1) * ldc
    __device__ __forceinline__ int base(int X, int b) const { return (X ^ flip(X) ^ b) * ldc + c; }
};
struct RowLayout {              // one transform per padded row: a pad element
    int base;                   // after every 16 keeps the strides of the
    __device__ __forceinline__ int operator()(int row) const { return base + row + (row >> 4); }
};                              // stage exchanges free of bank conflicts

// Writes stage S's outputs to shared memory.
template <int L, int S, bool REV, typename C, class LAY>
__device__ __forceinline__ void store_stage(C *sm, const LAY &lay, int t, const C *v) {
    constexpr int R = radix(L, S, REV);
#pragma unroll
    for (int kk = 0; kk < E / R; ++kk)
#pragma unroll
        for (int r = 0; r < R; ++r) sm[lay(out_row<L, S, REV>(t, kk, r))] = v[kk * R + r];
}
// Reads stage S's inputs from shared memory.
template <int L, int S, bool REV, typename C, class LAY>
__device__ __forceinline__ void load_stage(const C *sm, const LAY &lay, int t, C *v) {
    constexpr int R = radix(L, S, REV);
#pragma unroll
    for (int kk = 0; kk < E / R; ++kk)
#pragma unroll
        for (int r = 0; r < R; ++r) v[kk * R + r] = sm[lay(in_row<L, S, REV>(t, kk, r))];
}
// The stage exchanges with ColLayoutHalf (t < TPC): a store of stage S
// writes row X | K with X = (t / Ns) Ns R + t mod Ns, K = kk TPC R + r Ns
// (Ns divides TPC in every stage that stores); a load reads X = t,
// K = kk TPC + r L/R.
template <int L, int S, bool REV, typename C>
__device__ __forceinline__ void store_stage(C *sm, const ColLayoutHalf &lay, int t, const C *v) {
    constexpr int R = radix(L, S, REV), Ns = stride_before(L, S, REV), TPC = L / E;
    static_assert(TPC % Ns == 0, "a stage that stores has Ns dividing TPC");
    const int X = (t / Ns) * Ns * R + t % Ns;
    const int b0 = lay.base(X, 0), b1 = lay.base(X, 1);
#pragma unroll
    for (int kk = 0; kk < E / R; ++kk)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int K = kk * TPC * R + r * Ns;
            sm[((ColLayoutHalf::flip(K) ^ (K & 1)) ? b1 : b0) + (K & ~1) * lay.ldc] = v[kk * R + r];
        }
}
template <int L, int S, bool REV, typename C>
__device__ __forceinline__ void load_stage(const C *sm, const ColLayoutHalf &lay, int t, C *v) {
    constexpr int R = radix(L, S, REV), TPC = L / E;
    const int b0 = lay.base(t, 0), b1 = lay.base(t, 1);
#pragma unroll
    for (int kk = 0; kk < E / R; ++kk)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int K = kk * TPC + r * (L / R);
            v[kk * R + r] = sm[((ColLayoutHalf::flip(K) ^ (K & 1)) ? b1 : b0) + (K & ~1) * lay.ldc];
        }
}
template <int L, int S, bool REV, typename C>
__device__ __forceinline__ void store_stage(C *sm, int ldc, int c, int t, const C *v) {
    store_stage<L, S, REV>(sm, ColLayout{ldc, c}, t, v);
}
template <int L, int S, bool REV, typename C>
__device__ __forceinline__ void load_stage(const C *sm, int ldc, int c, int t, C *v) {
    load_stage<L, S, REV>(sm, ColLayout{ldc, c}, t, v);
}

// Exchange from a radix-16 stage to a closing radix-2 stage (plans
// ..., 16, 2) when a transform's TPC threads are the consecutive lanes
// t = lane % TPC of one warp.  Register r of thread t holds row
// 16 Ns (t / Ns) + t % Ns + r Ns (Ns = TPC / 2); the radix-2 stage wants in
// register 2k + b of thread t' the row t' + k TPC + b L/2.  So thread t keeps
// its registers of parity t / Ns and trades the other eight with thread
// t ^ Ns: sixteen warp shuffles per thread instead of a round trip through
// shared memory.
template <int L, typename C> __device__ __forceinline__ void swap_exchange(C *v, int t) {
    constexpr int NS2 = L / 32;   // partner distance (the radix-16 stage's Ns)
    const bool lo = (t & NS2) == 0;
#pragma unroll
    for (int k = 0; k < E / 2; ++k) {
        const C a = v[2 * k], b = v[2 * k + 1];
        C snd, rcv;
        snd.x = lo ? b.x : a.x;
        snd.y = lo ? b.y : a.y;
        rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, NS2);
        rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, NS2);
        v[2 * k].x = lo ? a.x : rcv.x;
        v[2 * k].y = lo ? a.y : rcv.y;
        v[2 * k + 1].x = lo ? rcv.x : b.x;
        v[2 * k + 1].y = lo ? rcv.y : b.y;
    }
}

// Registers of a forward transform's last stage (natural-order rows) renamed
// to the first stage of the same (unreversed) plan: an inverse transform
// with the forward plan starts from the forward outputs without an
// exchange.  Last stage radix RL: register kk*RL + q holds row
// t + kk TPC + q L/RL, which is row t + (kk + q E/RL) L/16 of the radix-16
// first stage.
template <int L, typename C> __device__ __forceinline__ void regs_last_to_first(C *v) {
    constexpr int RL = radix(L, nstages(L) - 1, false);
    C u[E];
#pragma unroll
    for (int kk = 0; kk < E / RL; ++kk)
#pragma unroll
        for (int q = 0; q < RL; ++q) u[kk + q * (E / RL)] = v[kk * RL + q];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = u[e];
}
// An inverse transform of length L whose input comes from the forward's
// registers runs the forward (unreversed) plan when that plan closes with a
// radix-2 stage: its exchanges are then one through shared memory and one
// by shuffles (swap_exchange), against two through shared memory for the
// reversed plan.
__host__ __device__ constexpr bool inv_fwd_plan(int L) { return nstages(L) > 1 && fwd_radix(L, nstages(L) - 1) == 2; }

// Runs stages 0..NS-1 given stage 0's inputs in registers; exchanges through
// shared memory (layout lay) between stages.  On return the registers hold
// the last stage's outputs (natural order rows in_row of the last stage).
// All threads of the block must call it (it synchronises).
// ZIN: the inputs of rows >= L/2 are zero (forward transforms of padded
// data; the first stage is radix 16 and only registers r < 8 are read).
// HOUT: only the outputs of rows < L/2 are used (inverse transforms: a
// radix-16 last stage keeps registers r < 8, a closing radix-2 stage its
// registers 2k).
// WSYNC: a transform's TPC threads are the consecutive lanes t = lane % TPC
// of one warp and its exchange area is touched by that warp only, so the
// exchanges synchronise the warp instead of the block, and an exchange into
// a closing radix-2 stage goes by warp shuffles (swap_exchange).
template <bool WSYNC> __device__ __forceinline__ void xsync() {
    if (WSYNC) __syncwarp(); else __syncthreads();
}
template <int L, bool REV, int SIGN, bool ZIN = false, bool HOUT = false, bool WSYNC = false, typename C, class LAY>
__device__ __forceinline__ void fft_core(C *v, C *sm, const LAY &lay, int t, const C *tw) {
    constexpr int NS = nstages(L);
    stage_butterflies<L, 0, REV, SIGN, ZIN, HOUT && NS == 1>(v, t, tw);
    if (NS > 1) {
        if constexpr (WSYNC && NS == 2 && radix(L, 0, REV) == 16 && radix(L, NS - 1, REV) == 2) {
            swap_exchange<L>(v, t);
        } else {
            store_stage<L, 0, REV>(sm, lay, t, v);
            xsync<WSYNC>();
            load_stage<L, (NS > 1 ? 1 : 0), REV>(sm, lay, t, v);
            xsync<WSYNC>();
        }
        stage_butterflies<L, (NS > 1 ? 1 : 0), REV, SIGN, false, HOUT && NS == 2>(v, t, tw);
    }
    if (NS > 2) {
        if constexpr (WSYNC && radix(L, 1, REV) == 16 && radix(L, NS - 1, REV) == 2) {
            swap_exchange<L>(v, t);
        } else {
            store_stage<L, (NS > 1 ? 1 : 0), REV>(sm, lay, t, v);
            xsync<WSYNC>();
            load_stage<L, (NS > 2 ? 2 : 0), REV>(sm, lay, t, v);
            xsync<WSYNC>();
        }
        stage_butterflies<L, (NS > 2 ? 2 : 0), REV, SIGN, false, HOUT>(v, t, tw);
    }
}
template <int L, bool REV, int SIGN, bool ZIN = false, bool HOUT = false, typename C>
__device__ __forceinline__ void fft_core(C *v, C *sm, int ldc, int c, int t, const C *tw) {
    fft_core<L, REV, SIGN, ZIN, HOUT>(v, sm, ColLayout{ldc, c}, t, tw);
}

}  // namespace pmfft
