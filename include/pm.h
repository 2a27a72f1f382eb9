/*
 * pm.h - C ABI of the GB300 nested-grid particle-mesh gravity step
 *        (Superbox-10: Bien, Brandt & Just 2012, MNRAS).
 *
 * One step of the method (Sec. 2.1 and 2.2 of the paper), per galaxy and per
 * grid level (grids 1-5: fine, medium x2, coarse x2):
 *   recentre grids 1-3, assign mass to cells (Eq. eqn:cell), zero-pad to the
 *   doubled isolated-boundary grid, forward 3D real FFT, multiply by the
 *   precomputed Green's function H-hat (Eq. eqn:greens, eq:symmetry), inverse
 *   FFT (Eq. eq:poisson evaluated exactly), finite-difference forces with
 *   first-order Taylor interpolation (Eq. eqn:diff) summed by the potential
 *   combination rule, and the leap-frog kick-drift.
 *
 * Conventions shared by every call:
 *   - Units: Phi = +G sum rho H is positive; the acceleration is +grad Phi.
 *   - Grid arrays are laid out [z][y][x] with x fastest.
 *   - Particle arrays are device memory owned by the caller, structure of
 *     arrays, float for PM_FP32 contexts and double for PM_FP64 contexts.
 *   - Every call is asynchronous on the context's stream (pm_set_stream)
 *     unless stated; only the pm_get_* and pm_diagnostics calls synchronise.
 *   - Every call returns PM_OK (0) or a negative PM_E_* status and never
 *     throws; pm_last_error() gives a message for the calling thread.
 *   - Particles flagged lost (PM_FLAG_LOST) contribute nothing and are not
 *     moved; the flag is set by pm_deposit and never cleared by the library.
 */
#ifndef PM_H
#define PM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_OK           0
#define PM_E_ARG       -1   /* invalid argument, size or pointer            */
#define PM_E_QCRIT     -2   /* medium-grid flattening below q_crit          */
#define PM_E_NESTING   -3   /* grid 1 not inside grid 2, or grid 2 not inside grid 4 */
#define PM_E_OVERFLOW  -4   /* mass bound leaves no fixed-point headroom    */
#define PM_E_CUDA      -5   /* a CUDA runtime call failed                   */
#define PM_E_STATE     -6   /* call not valid in the context's state        */
#define PM_E_TIMEOUT   -7   /* a kernel's bounded wait for a tensor copy expired
                               (reported by the next synchronising call)     */

#define PM_FP32 1
#define PM_FP64 2

#define PM_FLAG_LOST 1u

#define PM_MAX_GALAXIES 8

typedef struct pm_ctx pm_ctx;

/* One grid (Sec. 2.1, Eq. eqn:cell; flattening Sec. 2.2.2): nx*ny*nz active
 * cells, each a power of two in [8, 256]; cell lengths l_xy (x and y) and
 * l_z = q*l_xy.  A geometry with nx == 0 is absent. */
typedef struct {
    int32_t nx, ny, nz;
    double  l_xy, l_z;
} pm_geometry;

/* One galaxy's grids (Sec. 2.1): fine = grid 1, medium = grids 2 and 3,
 * coarse = grids 4 and 5.  Grids 1-3 are centred on `centre` and, when
 * `recentre` is nonzero, move each step to the centre of mass of the
 * galaxy's live particles within r_core of the previous centre.  Grids 4-5
 * are centred on the system centre.  Regions: core r < r_core (and inside
 * grids 1 and 2), shell r < r_out (inside grid 2), outer otherwise.  A galaxy
 * without medium grid has only grid 5 (a plain single-grid PM). */
typedef struct {
    pm_geometry coarse, medium, fine;
    double  r_core, r_out;
    double  centre[3];
    int32_t recentre;
} pm_galaxy;

/* The whole system.  Particles farther than r_sys from sys_centre, or outside
 * the usable box (two empty boundary cells, Sec. 2.1) of any coarse grid,
 * are lost.  mass_bound >= sum |m| fixes the 64-bit fixed-point mass scale
 * 2^s with s = 62 - ceil(log2(mass_bound)).  h000 is the Green's function
 * self-term H(0,0,0) in units of 1/l_xy (the paper leaves it open; 1 gives
 * zero self-force on cubic cells). */
typedef struct {
    int32_t precision;           /* PM_FP32 or PM_FP64                     */
    int32_t ngal;                /* 1 .. PM_MAX_GALAXIES                   */
    double  G, h000, r_sys;
    double  sys_centre[3];
    double  mass_bound;
} pm_system;

/* Caller-owned device arrays (pointers to float or double per precision). */
typedef struct {
    void *x, *y, *z, *vx, *vy, *vz, *m;
    const int32_t *gal;          /* galaxy index of each particle          */
    uint32_t *flags;             /* bit 0: lost                            */
    int64_t n;                   /* number of particles, >= 0              */
} pm_particles;

/* Host helpers (no GPU needed). */
/* Cell length of a grid whose N-4 usable cells span 2R, flattened by q
 * (Sec. 2.1 boundary cells; Sec. 4.1 Table 3): 2 R q / (N - 4). */
double pm_cell_length(double R, int32_t N, double q);
/* Smallest admissible flattening of grids 2-3 (Sec. 2.2.2):
 * max(R_core/R_out, 4/(N-4) * R_sys/R_out). */
double pm_q_crit(double r_core, double r_out, double r_sys, int32_t N);
/* Fixed-point shift s for a mass bound, or INT32_MIN if the bound is not
 * positive and finite. */
int32_t pm_fixed_shift(double mass_bound);
/* Message of the last failing call on this thread ("" if none). */
const char *pm_last_error(void);

/* Builds every grid, its H-hat table (FP64 on the device, stored in the
 * context precision) and all work buffers on the current CUDA device.
 * `stream` is a cudaStream_t (NULL = legacy default stream) on which later
 * calls are ordered.  Validates: powers of two, q >= q_crit for flattened
 * medium grids (PM_E_QCRIT), grid 1 inside grid 2 inside grid 4
 * (PM_E_NESTING), galaxies after the first not flattened (Sec. 2.2.2).
 * Synchronises once.  *out is NULL on failure. */
int pm_create_grids(const pm_system *sys, const pm_galaxy *gals, void *stream,
                    pm_ctx **out);
void pm_destroy(pm_ctx *ctx);
int pm_set_stream(pm_ctx *ctx, void *stream);

/* Step a1 (Sec. 2.1 recentring): move grids 1-3 of recentring galaxies to
 * the centre of mass of their live particles within r_core (exact integer
 * accumulation, order independent). */
int pm_recentre(pm_ctx *ctx, const pm_particles *p);

/* Step a1 split for a step whose particles are sharded across processes
 * (one GPU each): pm_recentre_sums adds the exact integer centre-of-mass
 * sums of this process's particles into the context's accumulators (the
 * csum buffer of pm_exchange_buffers); after the caller has summed that
 * buffer across processes (integer sums: exact, order independent),
 * pm_recentre_apply moves the centres from the summed accumulators and
 * zeroes them.  pm_recentre is both in one call. */
int pm_recentre_sums(pm_ctx *ctx, const pm_particles *p);
int pm_recentre_apply(pm_ctx *ctx);

/* Device buffers that a sharded step sums across processes (Sec. 2.1
 * grids; Sec. 2.2.3 parallelises the paper's own solver): rho = every mass
 * set's int64 density, one contiguous block of *rho_bytes bytes, filled by
 * pm_deposit with this process's particles; csum = the centre-of-mass
 * accumulators (int64, *csum_bytes bytes).  Element-wise int64 sums of
 * these buffers over the processes give exactly the single-process
 * densities and centres.  The pointers belong to the context. */
int pm_exchange_buffers(pm_ctx *ctx, void **rho, int64_t *rho_bytes, void **csum, int64_t *csum_bytes);

/* Steps a8-a9 with the potentials of the last pm_solve (Sec. 2.1 leap-frog):
 * v += dt a(x); x += dt v, for this process's particles. */
int pm_kick_drift(pm_ctx *ctx, const pm_particles *p, double dt);

/* Steps a2-a3 (Eq. eqn:cell, Sec. 2.1 grids 1-5, Sec. 2.2.1 individual
 * masses): classify every particle, set lost flags, and add its fixed-point
 * mass to the int64 density of each grid it belongs to.  Densities are
 * zeroed first; the result is bit-exact and independent of thread order. */
int pm_deposit(pm_ctx *ctx, const pm_particles *p);

/* Steps a4-a7 (Sec. 2.1): for every grid, zero-pad, forward real 3D FFT,
 * multiply by H-hat, inverse FFT, keep the active region -> Phi.  Grid 1
 * (the fine grid) is also solved for the forward differences of Phi_1
 * along x, y and z (its spectrum times H-hat (e^{2 pi i k/L} - 1) per axis,
 * the same discrete values as differencing Phi_1), which pm_force uses for
 * Eq. eqn:diff on that grid; Phi_1 itself is kept as well.  Enqueued on the
 * context's stream, in the launch configuration pm_info reports. */
int pm_solve(pm_ctx *ctx);

/* Step a8 (Eq. eqn:diff + combination rule): acceleration of each particle
 * into caller-owned device arrays ax, ay, az (zero for lost particles).
 * Uses the potentials of the last pm_solve. */
int pm_force(pm_ctx *ctx, const pm_particles *p, void *ax, void *ay, void *az);

/* v += dt * a with a from the last pm_solve (leap-frog start: dt = -dt0/2). */
int pm_kick(pm_ctx *ctx, const pm_particles *p, double dt);

/* Steps a1-a9, nsteps times: recentre, deposit, solve, force and leap-frog
 * kick-drift (Sec. 2.1): v(t+dt/2) = v(t-dt/2) + dt a(t);
 * x(t+dt) = x(t) + dt v(t+dt/2).  The step is captured as CUDA graphs per
 * (particle arrays, n, dt) and replayed; the graphs of the four most
 * recently stepped particle sets are kept (the least recently used is
 * replaced), so a caller may alternate buffers without recapturing. */
int pm_step(pm_ctx *ctx, const pm_particles *p, double dt, int32_t nsteps);

/* Step a10 (energy and angular momentum, Sec. 6.4 quantities): recentre is
 * not applied; deposit + solve at the current positions, then with
 * v(t) = v(t-dt/2) + dt/2 a(t): out[0] = K = sum m v^2/2, out[1] = W =
 * -1/2 sum m Phi(x), out[2] = K + W, out[3..5] = L = sum m x cross v,
 * out[6] = number of live particles.  FP64 sums.  Synchronises. */
int pm_diagnostics(pm_ctx *ctx, const pm_particles *p, double dt, double *out);

/* Test and inspection hooks (synchronise).  set = 1..5 as in the paper.
 * pm_get_potential returns the potentials as the force stencils combine
 * them: set 1 Phi_1, set 2 Phi_2 + Phi_3, set 3 Phi_3, set 4 Phi_4 + Phi_5,
 * set 5 Phi_5. */
int pm_get_density(pm_ctx *ctx, int32_t gal, int32_t set, int64_t *host_out);
int pm_get_potential(pm_ctx *ctx, int32_t gal, int32_t set, void *host_out);
int pm_get_centres(pm_ctx *ctx, double *host_out);          /* ngal*3 */
int pm_set_centres(pm_ctx *ctx, const double *host_in);     /* ngal*3 */
int pm_count_lost(pm_ctx *ctx, const pm_particles *p, int64_t *host_out);
/* host_out[6] = [fixed-point shift, mass sets, distinct geometries, device
 * bytes, solve schedule, batched].  The solve's schedule is chosen when the
 * context is created by timing each on the device.  Its units are either the
 * grid shapes (batched = 1: the pairs of mass sets of every geometry of one
 * shape, e.g. the same-size grids of several galaxies, share each FFT pass's
 * launches) or the single geometries (batched = 0: a launch per pair); their
 * chains of passes run as 0 = one branch stream per unit, all starting
 * together; 1 = two branch streams of about equal work, one running its
 * chains largest first and the other smallest first; -1 = a single unit (no
 * branches). */
int pm_info(pm_ctx *ctx, int64_t *host_out);

/* Sets the solve's launch configuration in place of the one chosen by timing
 * at creation: batched (1: the pairs of one grid shape share each pass's
 * launches; 0: a launch per pair) and schedule (0: one branch stream per
 * unit; 1: two staggered lanes; ignored with a single unit).  Every
 * configuration computes the same results bit for bit (the same arithmetic
 * per pair; only the launch grouping and the stream order differ).  Waits
 * for the context's stream and drops its captured step graphs.  PM_E_ARG
 * for values other than 0 and 1. */
int pm_set_launch_config(pm_ctx *ctx, int32_t batched, int32_t schedule);

/* Self-test of failure detection (no counterpart in the paper): launches one
 * block that waits, with the bounded wait the FFT passes use for their
 * tensor copies (2 s limit), on a barrier that nothing arrives at.  The wait
 * gives up, the block sets the context's device error flag, and the call
 * returns what the next synchronising call reports after an expired wait of
 * a pass: PM_E_TIMEOUT.  The flag is cleared afterwards, so the context stays
 * usable.  Takes about two seconds; synchronises.  PM_E_TIMEOUT from this
 * call is the expected result, not a failure. */
int pm_selftest_wait_expiry(pm_ctx *ctx);

/* Spatial sort (no counterpart in the paper; a locality optimisation of the
 * NGP assignment of Eq. eqn:cell): permutes every particle array of p in
 * place so that particles are ordered by galaxy, region (core, shell,
 * outer) and cell of that region's grid (cells binned so a grid has at most
 * 2^21 bins); lost particles go last.  Order within a cell is unspecified.
 * If perm is not NULL (device int64[n]) it receives perm[new] = old.
 * Results of the step do not depend on the order.  Allocates its scratch
 * (about 44 bytes per particle) on first use. */
int pm_sort(pm_ctx *ctx, const pm_particles *p, int64_t *perm);
/* pm_step re-sorts the particles before every k-th step (k = 0: never, the
 * default); resets the step counter so the next step sorts. */
int pm_set_sort_interval(pm_ctx *ctx, int32_t k);

/* Per-phase device time of the next `nsteps` steps, run without the graph,
 * with CUDA events on the context's launch stream between phases:
 * ms_out[0] recentre, [1] deposit (incl. zeroing), [2] x forward pass,
 * [3] y forward pass, [4] z pass (forward, H-hat multiply, inverse),
 * [5] y inverse pass, [6] x inverse pass, [7] force + kick-drift,
 * [8] whole steps, [9] spatial sort (steps where it is due); each the total
 * over the steps (ms_out holds 10 floats).  Synchronises. */
int pm_step_timed(pm_ctx *ctx, const pm_particles *p, double dt, int32_t nsteps,
                  float *ms_out);

/* ---- CIC variant for differentiable runs ------------------------------
 * Not the paper's scheme: nearest-grid-point assignment (Eq. eqn:cell) has
 * zero position gradient almost everywhere, so gradients of trajectories use
 * cloud-in-cell instead.  Each particle spreads its mass over the 8 cells
 * around it with trilinear weights W; the grid field is the central
 * difference of the potential (the first term of Eq. eqn:diff) at every
 * cell; the acceleration is that field interpolated with the same weights.
 * Regions, mass sets, the convolution and the combination rule (Sec. 2.1)
 * are those of the NGP step; the grid centres are not moved (no recentring),
 * so they are constants of the map.  The lower CIC cell along an axis is
 * a - 1 (fraction t + 1) when t = Delta/l < 0, else a (fraction t), with a
 * the NGP cell and Delta the offset from its centre.  Enqueued on the
 * context's stream unless stated otherwise.
 *
 * pm_cic_deposit: lost test as pm_deposit, then int64 fixed-point CIC mass
 * (each of the 8 cell shares rounded separately) into the five sets.  Use
 * pm_solve afterwards.
 * pm_cic_force: ax, ay, az (device, context precision, n) = CIC acceleration
 * from the current potentials; lost particles get 0.
 * pm_cic_kick_drift: v += dt_kick a; x += dt_drift v (live particles).
 * pm_cic_vjp: vector-Jacobian product of the CIC acceleration at the
 * current positions and masses, whose potentials must be the current ones
 * (pm_cic_deposit + pm_solve at these positions): with u = (ux, uy, uz) one
 * cotangent per particle, adds u^T da/dx to (gx, gy, gz) and u^T da/dm to
 * gm (device arrays, context precision, n; caller-owned, accumulated into).
 * Both the particle's own interpolation weights and, through the
 * (symmetric) convolution, every other particle's mass assignment
 * contribute.  The adjoint densities are int64 fixed point with a scale
 * chosen from max |u| (one device-to-host read; the call synchronises), so
 * the result does not depend on the order of the atomics.  Afterwards the
 * density and potential buffers hold adjoint fields: deposit and solve again
 * before the next force.  PM_E_ARG for a non-finite cotangent. */
int pm_cic_deposit(pm_ctx *ctx, const pm_particles *p);
int pm_cic_force(pm_ctx *ctx, const pm_particles *p, void *ax, void *ay, void *az);
int pm_cic_kick_drift(pm_ctx *ctx, const pm_particles *p, double dt_kick, double dt_drift);
int pm_cic_vjp(pm_ctx *ctx, const pm_particles *p, const void *ux, const void *uy, const void *uz,
               void *gx, void *gy, void *gz, void *gm);

/* ---- disc diagnostics (Sec. 6 quantities) ------------------------------
 * FP64 reductions over the selected particles that are not lost: select
 * (device uint8[n], nonzero = take) or NULL for every particle of galaxy
 * q->gal.  Positions and velocities are taken relative to the current grid
 * centre of galaxy q->gal (x, y in the disc plane); velocities are the
 * stored ones (v(t - dt/2) inside a run: kick by dt/2 first to synchronise).
 * With R = |(dx, dy)|, phi = atan2(dy, dx), v_R, v_phi the cylindrical
 * components:
 *   bins: q->nbins (1..64) radial bins of equal particle numbers, bounded
 *     by the exact order statistics of R^2 at ranks floor(k n / nbins),
 *     k = 1..nbins-1 (a particle is in bin #{k : edge_k <= R^2});
 *   E_heat = sum m |v - vbar_c(R) e_phi|^2 / 2, vbar_c linear in R between
 *     the bins' (mean R, mean v_phi) and constant beyond (Sec. 6 heat);
 *   annulus q->r0 - q->dr <= R < q->r0 + q->dr: mass-weighted sigma_R,
 *     sigma_phi, sigma_z (Sec. 6 dispersion ratio);
 *   rings: q->nring rings of width q->r_ring / q->nring from R = 0 (R > 0),
 *     A~_m = (1/S) sum m_j exp(-i m phi_j), m = 1..q->mmax, S the ring area
 *     (Sec. 6 Fourier modes); nring * mmax <= 1024.
 * out (host, 6 + 4 nbins + 2 nring mmax doubles): [n, E_heat, sigma_R,
 * sigma_phi, sigma_z, annulus mass, then per bin (mean R, count,
 * sqrt<z^2>, mean v_phi), then per ring and mode (Re A~_m, Im A~_m)].
 * Synchronises (the bin edges take 8 radix passes with a host step each);
 * allocates 0.1 MB of scratch on the first call. */
typedef struct {
    int32_t gal;
    int32_t nbins;
    int32_t nring;
    int32_t mmax;
    double r_ring;
    double r0, dr;
} pm_disc_query;
int pm_disc_diagnostics(pm_ctx *ctx, const pm_particles *p, const uint8_t *select,
                        const pm_disc_query *q, double *out);

/* Allocation-free potential of one isolated grid.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (a host application whose device memory is pre-partitioned by
 * its own pool, where a cudaMalloc fails or synchronises the device; a
 * plugin that may not allocate after start-up).
 *
 * Computes what pm_solve computes for one grid: Phi = G/l_xy * (rho * H) on
 * the nx*ny*nz active region of the doubled grid, with H-hat rebuilt in FP64
 * on every call.  rho: device int64 density, layout [z][y][x], mass per cell
 * in units of 2^-shift (the fixed point of pm_deposit); phi: device output,
 * float (precision PM_FP32) or double (PM_FP64), same layout.  Both are the
 * caller's.  Work is enqueued on `stream` (a cudaStream_t, NULL = legacy
 * default stream); the call returns without waiting for it.
 *
 * Scratch: every intermediate lives in one file-scope device array of
 * 32 MiB that each GPU loading the library holds until the process exits;
 * the call allocates and frees nothing.  A grid whose intermediates exceed
 * 32 MiB is refused with PM_E_ARG (e.g. 64^3 in FP64 and 128x128x32 in FP32
 * fit; 128^3 does not).  All calls on a device share the array and it keeps
 * the previous call's contents; each call writes every scratch value before
 * reading it, so nothing needs clearing, but calls whose work overlaps on the
 * GPU (different streams, or other threads) race on it and must be ordered
 * by the caller.  Every call looks up the array's device address (a host-side
 * lookup) and the first call on a device and precision also sets kernel
 * attributes.
 *
 * Failure of a bounded wait: a pass whose tensor copy does not complete
 * within its time limit stops early; the call's last kernel then fills phi
 * with NaN and raises a status word of the device, which
 * pm_potential_static_status reports. */
int pm_potential_static(const int64_t *rho, void *phi, int32_t nx, int32_t ny, int32_t nz,
                        double l_xy, double l_z, double G, double h000, int32_t shift,
                        int32_t precision, void *stream);

/* Status of the allocation-free calls on the current device (no counterpart
 * in the paper): waits for `stream`, then returns PM_E_TIMEOUT if a
 * pm_potential_static call since the last status query had an expired wait
 * (its phi holds NaN), else PM_OK; the status word is cleared by the query.
 * Allocates nothing; synchronises. */
int pm_potential_static_status(void *stream);

/* Self-test of that failure report (no counterpart in the paper): one block
 * waits, with the bounded wait of the passes (2 s), on a barrier nothing
 * arrives at, and sets the error word of the static scratch; the same last
 * kernel as pm_potential_static then fills phi (n values, float or double
 * per precision) with NaN and raises the status word.  Enqueued on `stream`;
 * pm_potential_static_status then returns PM_E_TIMEOUT. */
int pm_static_selftest_wait_expiry(void *phi, int64_t n, int32_t precision, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PM_H */
