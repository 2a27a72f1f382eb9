// Launch interface between the C ABI (pm_api.cu) and the kernels, which are
// instantiated per precision in pm_fp32.cu and pm_fp64.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include "pm_internal.cuh"

// One FFT pass over a pair of mass sets of one geometry packed as
// rho_a + i rho_b (rho_b may be null).
struct PairArgs {
    const long long *rho_a, *rho_b;       // int64 densities [z][y][x]
    void *work;                           // complex [nz][2ny][2nx]
    void *phi_b;                          // Phi_b (null without partner)
    void *phi_sum;                        // Phi_a + Phi_b (or Phi_a)
    const void *hhat;                     // H-hat octant [nz+1][ny+1][nx+1]
    const void *tw;                       // exp(-2 pi i m / L), m < L, this pass's L
    int nx, ny, nz;
    double scale;                         // 2^-s
    int *err;                             // 1: a tensor copy never completed; 2: an unsupported launch
    // Difference fields of an unpaired grid (rho_b null).  D_L(k) =
    // exp(2 pi i k / L) - 1 multiplies the spectrum of a field f into that of
    // its forward difference f[n+1] - f[n]; dtx, dty, dtz are tables of D for
    // the x, y and z lengths.  dmode (z pass): 0 multiplies by H-hat,
    // 1 by H-hat (D_x + i D_y), 2 by H-hat (D_z + i); the inverse of a real
    // field's spectrum times such a factor is fx + i fy, or fz + i Phi.
    // 3: both from one forward transform (L <= 64, H-hat from the
    // thread-major table; L = 128 and 256 when the tile's H-hat rows are
    // staged, COLS <= nx): fx + i fy through smap, then fz + i Phi in place
    // through lmap.
    const void *dtx, *dty, *dtz;
    int dmode;
    int split;                            // x inverse: phi_sum = Re, phi_b = Im (no sum)
};

enum { COL_YFWD = 0, COL_ZCONV = 1, COL_YINV = 2 };

// One launch of an FFT pass over up to PM_BATCH items: work arrays of the
// same shape (nx, ny, nz), e.g. the grids of the same size of every galaxy
// (Sec. 2.1: all galaxies use the same kinds of grid).  Each item has its own
// arrays, H-hat table and tensor maps (lmap: the column passes' loads; smap:
// their stores); the launch walks the items' tiles (or x-pass row
// groups) as one index space, 2^lgi per item (set by the launcher).
#ifndef PM_BATCH
#define PM_BATCH 8
#endif
struct PassBatch {
    CUtensorMap lmap[PM_BATCH];
    CUtensorMap smap[PM_BATCH];
    PairArgs a[PM_BATCH];
    int n;
    int lgi;
};

// Columns per tile of the column passes for transform length L and real
// size esz: 16 threads per column, 256 threads per block, and a tensor-map
// box row of at most 256 eight-byte elements.
__host__ __device__ constexpr int pm_col_cols(int L, int esz) {
    return (4096 / L) < (esz == 4 ? 256 : 128) ? (4096 / L) : (esz == 4 ? 256 : 128);
}

// Columns per swizzled sub-tile of the z pass: as many as fill a 128-byte
// shared-memory row (16 FP32 or 8 FP64 complex values), at most a tile.
__host__ __device__ constexpr int pm_zsub_cols(int L, int esz) {
    return pm_col_cols(L, esz) < (esz == 4 ? 16 : 8) ? pm_col_cols(L, esz) : (esz == 4 ? 16 : 8);
}

// Tensor maps (2D, 8-byte elements) of one pair's work array for the
// column passes: y forward (box pm_col_cols columns x min(ny,256) rows), y
// inverse (box rows min(2ny,256)), z (box pm_zsub_cols columns x
// min(nz,256) rows, swizzled to the box row width; the z pass's loads and
// stores).  Host only; no device memory is touched.
int pm_encode_col_maps(void *work, int nx, int ny, int nz, int esz, CUtensorMap *yfwd, CUtensorMap *yinv,
                       CUtensorMap *zmap);

template <typename T> cudaError_t pm_set_attrs();
// Batched passes: x forward, column pass `mode` (y forward: loads through
// the items' yfwd maps, stores through their yinv maps, whose boxes hold
// the 2ny output rows; y inverse: loads through yinv, stores through yfwd
// (ny rows kept); z: loads through lmap and stores through smap, the same
// map in place or another work array's for the first difference-field
// pass), x inverse.  Every item of a batch has the same shape, precision
// and, in the z pass, dmode.
template <typename T> cudaError_t pm_launch_xfwd(PassBatch b, cudaStream_t st);
template <typename T> cudaError_t pm_launch_col(PassBatch b, int mode, cudaStream_t st);
template <typename T> cudaError_t pm_launch_xinv(PassBatch b, cudaStream_t st);
// A batch of one item (a pair's arrays and its maps; smap = lmap if null).
PassBatch pm_single_batch(const PairArgs &a, const CUtensorMap *lmap, const CUtensorMap *smap);

template <typename T>
cudaError_t pm_launch_deposit(const PartK<T> &p, const SysK &sk, const CenK *cen, int aggregate, cudaStream_t st);
// mode: 0 kick-drift, 1 write accelerations, 2 kick only, 3 diagnostics
template <typename T>
cudaError_t pm_launch_force(int mode, const PartK<T> &p, const SysK &sk, const CenK *cen, double dt,
                            T *ax, T *ay, T *az, double *diag, cudaStream_t st);
// Recentring from the current positions (part: zeroed accumulators).
// phase bit 0: add the particles' integer centre-of-mass sums into part;
// bit 1: add part's rows, move the centres and zero part again.
template <typename T>
cudaError_t pm_launch_recentre(const PartK<T> &p, const SysK &sk, CenK *cen, long long *part, int phase,
                               cudaStream_t st);
template <typename T>
cudaError_t pm_launch_count_lost(const PartK<T> &p, unsigned long long *out, cudaStream_t st);
// Counting sort by spatial key; permutes p's arrays in place through scratch.
template <typename T>
cudaError_t pm_launch_sort(const PartK<T> &p, const PartK<T> &scratch, const SysK &sk, const CenK *cen,
                           const SortK &so, unsigned *count, unsigned *key, unsigned *rank, unsigned *bsum,
                           long long *perm, cudaStream_t st);

// CIC variant (differentiable runs).  field modes: 0 kick (dtk) and drift
// (dtd), 1 write accelerations to o*, 2 add the direct term of the adjoint
// for cotangent u to o*, 3 spread u into the density slots as int64 with
// scale qs (adjoint densities).
template <typename T>
cudaError_t pm_launch_cic_deposit(const PartK<T> &p, const SysK &sk, const CenK *cen, cudaStream_t st);
template <typename T>
cudaError_t pm_launch_cic_field(int mode, const PartK<T> &p, const SysK &sk, const CenK *cen, double dtk, double dtd,
                                T *ox, T *oy, T *oz, const T *ux, const T *uy, const T *uz, double qs,
                                cudaStream_t st);
// Adds the field term of the adjoint (from the adjoint solve's potentials).
template <typename T>
cudaError_t pm_launch_cic_gather(const PartK<T> &p, const SysK &sk, const CenK *cen, T *gx, T *gy, T *gz, T *gm,
                                 cudaStream_t st);
// max |u| over live particles into *out (float bits, atomicMax; zero it first).
template <typename T>
cudaError_t pm_launch_cic_umax(const PartK<T> &p, const T *ux, const T *uy, const T *uz, unsigned *out,
                               cudaStream_t st);

// Disc diagnostics (Sec. 6 quantities): particle view and query.
namespace pmk {
template <typename T> struct DiagP {
    const T *x, *y, *z, *vx, *vy, *vz, *m;
    const uint32_t *flags;
    const uint8_t *sel;     // null: particles of galaxy `gal`
    const int32_t *gal_id;
    int gal;
    long long n;
    double c[3];
};

// Accumulator layout: per bin [sum R, count, sum z^2, sum v_phi]; annulus
// [M, M vR, M vR^2, M vphi, M vphi^2, M vz, M vz^2]; per ring and mode
// [sum m cos(m phi), -sum m sin(m phi)].
struct DiagQ {
    int nbins, nring, mmax;
    double width, r_ring, rlo, rhi;
};

}  // namespace pmk
// Radix-select pass over the bits of R^2 (pass 0..7), the sums of the bins,
// annulus and rings, and the heat about an interpolated circular velocity.
template <typename T> cudaError_t pm_launch_diag_hist(const pmk::DiagP<T> &d, int pass, const unsigned long long *pref,
                                                      int npref, unsigned *hist, cudaStream_t st);
template <typename T> cudaError_t pm_launch_diag_sums(const pmk::DiagP<T> &d, const pmk::DiagQ &q,
                                                      const unsigned long long *edges, double *acc, cudaStream_t st);
template <typename T> cudaError_t pm_launch_diag_heat(const pmk::DiagP<T> &d, const double *xp, const double *fp,
                                                      int np, double *acc, cudaStream_t st);

// FP64 H-hat construction (precision independent) and storage conversion.
cudaError_t pm_green_octant(double *h, int nx, int ny, int nz, double q, double h000, cudaStream_t st);
cudaError_t pm_axis_transform(const double *in, double *out, const double *cmat, int n1,
                              long long outer, long long inner, cudaStream_t st);
// H-hat table of the z pass from the FP64 octant oct[kzr][kyr][kxr]
// (scaled by `scale`): for each octant column (kyr, kxr), for L = 2nz >= 128
// the nz + 1 values H-hat(kzr) padded with zeros to pm_hhat_stride(L); for
// L <= 64 the L values H-hat(kz) (kz > L/2 mirrored) in thread-major order,
// register e of thread t at entry t * 16 + e (hhat_thread_major).
// For L = 2nz >= 128 each octant column holds only H-hat(kzr), kzr = 0..nz,
// padded to pm_hhat_stride(L) values: the smallest h >= nz + 1 with
// h = TPC (mod 2 TPC), TPC = L/16 threads per column, so that the columns of
// a warp (32/TPC of them) read disjoint shared-memory banks; each lane
// mirrors its kz itself.  Shorter transforms keep the full L values per
// column in thread-major order.
__host__ __device__ constexpr int pm_hhat_stride(int L) {
    return L < 128 ? L : (L / 16) + (L / 8) * ((L / 2 + 1 - L / 16 + L / 8 - 1) / (L / 8));
}
inline long long pm_hhat_table_size(int nx, int ny, int nz) {
    return (long long)(nx + 1) * (ny + 1) * pm_hhat_stride(2 * nz);
}
template <typename T>
cudaError_t pm_store_hhat(const double *oct, T *out, int nx, int ny, int nz, double scale, cudaStream_t st);

// Self-test of the bounded waits: one block waits on an mbarrier nothing
// arrives at, gives up after the time limit and sets *err to 1.
cudaError_t pm_launch_wait_expiry(int *err, cudaStream_t st);

// Records a message for pm_last_error() and returns code (C++ linkage; for
// translation units other than the C ABI file).
int pm_internal_fail(int code, const char *msg);
