// C ABI of the nested-grid particle-mesh step (declared in include/pm.h).
//
// The context owns every grid buffer: per galaxy and mass set an int64
// density, an FP32/FP64 spectrum work buffer ([z][y in 2ny][kx in nx+1]) and
// the potential; per distinct geometry the H-hat octant.  Particle arrays are
// the caller's.  All work is ordered on the caller's stream; pm_step replays a
// CUDA graph of one full step captured on a private stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pm.h"
#include "pm_launch.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define PM_CK(call)                                                                                  \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(PM_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                                   \
    } while (0)

#define PM_TRY(expr)               \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != PM_OK) return rc_; \
    } while (0)

bool pow2_in_range(int n) { return n >= 8 && n <= 256 && (n & (n - 1)) == 0; }

bool geom_present(const pm_geometry &g) { return g.nx != 0; }

bool geom_valid(const pm_geometry &g) {
    return pow2_in_range(g.nx) && pow2_in_range(g.ny) && pow2_in_range(g.nz) && std::isfinite(g.l_xy) &&
           std::isfinite(g.l_z) && g.l_xy > 0 && g.l_z > 0;
}

bool geom_equal(const pm_geometry &a, const pm_geometry &b) {
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.l_xy == b.l_xy && a.l_z == b.l_z;
}

// Half extent of the usable box along x/y and z: (n/2 - 2) l.
double ext_xy(const pm_geometry &g, int n) { return (n / 2 - 2) * g.l_xy; }
double ext_z(const pm_geometry &g) { return (g.nz / 2 - 2) * g.l_z; }

int ceil_log2(double v) {
    int e;
    double f = std::frexp(v, &e);
    return (f == 0.5) ? e - 1 : e;
}

GeomK make_geomk(const pm_geometry &g) {
    GeomK k;
    std::memset(&k, 0, sizeof(k));
    if (!geom_present(g)) return k;
    k.nx = g.nx; k.ny = g.ny; k.nz = g.nz;
    k.gxy = (float)(1.0 / g.l_xy);
    k.gz = (float)(1.0 / g.l_z);
    k.lxy = g.l_xy; k.lz = g.l_z;
    k.c_gx = 1.0 / (2.0 * g.l_xy);
    k.c_gz = 1.0 / (2.0 * g.l_z);
    k.c_hxx = 1.0 / (g.l_xy * g.l_xy);
    k.c_hzz = 1.0 / (g.l_z * g.l_z);
    k.c_mxy = 1.0 / (4.0 * g.l_xy * g.l_xy);
    k.c_mxz = 1.0 / (4.0 * g.l_xy * g.l_z);
    k.flxy = (float)k.lxy; k.flz = (float)k.lz;
    k.fc_gx = (float)k.c_gx; k.fc_gz = (float)k.c_gz;
    k.fc_hxx = (float)k.c_hxx; k.fc_hzz = (float)k.c_hzz;
    k.fc_mxy = (float)k.c_mxy; k.fc_mxz = (float)k.c_mxz;
    k.fil_xy = (float)(2.0 * k.c_gx); k.fil_z = (float)(2.0 * k.c_gz);
    return k;
}

// FP64 centres and their FP32 split c = hi + lo (hi = fl32(c), lo = fl32(c - hi)).
CenK make_cenk(const double *c, int ngal) {
    CenK k;
    std::memset(&k, 0, sizeof(k));
    for (int g = 0; g < ngal; ++g)
        for (int a = 0; a < 3; ++a) {
            k.c[g][a] = c[3 * g + a];
            k.hi[g][a] = (float)c[3 * g + a];
            k.lo[g][a] = (float)(c[3 * g + a] - (double)k.hi[g][a]);
        }
    return k;
}

// Captured steps for one particle set and time step: [0] step, [1] sort +
// step.  A context keeps a few such sets (e.g. the buffers of a caller that
// pipelines its copies) and replaces the least recently used.
struct GraphSet {
    bool valid = false;
    pm_particles key;
    double dt = 0;
    long long used = 0;
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
};
constexpr int GRAPH_SETS = 4;

// Two mass sets of one geometry transformed together as rho_a + i rho_b
// (b < 0: no partner), with their work array and tensor maps.
// A grid without partner (grid 1) is solved for its forward-difference
// fields instead (diff): the z pass runs twice, writing H-hat (D_x + i D_y)
// rho-hat into a second work array and H-hat (D_z + i) rho-hat in place, so
// that the inverse passes give fx + i fy and fz + i Phi.
struct Pair {
    int gi, a, b;
    bool diff = false;
    void *work = nullptr, *work2 = nullptr;
    CUtensorMap yfwd, yinv, zmap, yfwd2, yinv2, zmap2;
};

struct GeoBuf {
    pm_geometry g;
    long long A, workN, hatN;   // workN: complex elements of a pair's work array
    void *hhat = nullptr;
    std::vector<std::pair<int, int>> sets;   // (galaxy, set index 0..4)
    std::vector<Pair> pairs;
};

// Geometries of one shape (nx, ny, nz), e.g. the same-size grids of several
// galaxies: their pairs share each pass's launches (up to PM_BATCH pairs).
struct ShapeGroup {
    int nx, ny, nz;
    std::vector<int> geos;
};

}  // namespace

struct pm_ctx {
    pm_system sys;
    pm_galaxy gal[PM_MAX_GALAXIES];
    int prec = PM_FP32;
    size_t esz = 4;
    int shift = 0;
    double mscale = 1.0;
    std::vector<GeoBuf> geos;
    std::vector<ShapeGroup> shapes;
    // units of the solve's launches and branch streams: with `batched`, one
    // unit per shape whose pairs share each pass's launches; without, one
    // unit per geometry, each pair launched on its own (chosen by timing)
    bool batched = true;
    std::vector<std::vector<int>> units;   // geometry indices per unit
    int set_geo[PM_MAX_GALAXIES][PM_SETS];
    long long *rho[PM_MAX_GALAXIES][PM_SETS];
    void *phi[PM_MAX_GALAXIES][PM_SETS];
    void *fd[PM_MAX_GALAXIES][3];   // forward differences of Phi_1: fx, fy, fz (grid 1)
    long long *rho_all = nullptr;
    size_t rho_bytes = 0;
    SysK hs;
    SysK *d_sys = nullptr;
    CenK *d_cen = nullptr;
    long long *d_csum = nullptr;   // centre-of-mass accumulators (zero between uses)
    int *d_err = nullptr;          // set by a kernel whose bounded wait expired
    double *d_diag = nullptr;
    unsigned long long *d_cnt = nullptr;
    void *d_tw[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void *d_dt[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // exp(2 pi i k / L) - 1
    cudaStream_t user = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> branch;   // solve branch streams
    std::vector<cudaEvent_t> ev_join;
    // solve schedule, chosen by timing both at creation: 0 = one branch per
    // geometry, 1 = the geometries' chains in `lanes` (two branches)
    int sched = 0;
    std::vector<std::vector<int>> lanes;
    cudaEvent_t ev_fork = nullptr;
    GraphSet gs[GRAPH_SETS];
    long long guse = 0;
    // spatial sort
    SortK sortk;
    int sort_interval = 0;
    long long step_count = 0;
    long long sort_cap = 0;
    unsigned *s_count = nullptr, *s_key = nullptr, *s_rank = nullptr, *s_bsum = nullptr;
    void *s_arr[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t bytes = 0;
    std::vector<void *> allocs;
    bool any_recentre = false;
    // disc diagnostics scratch (allocated on first use)
    unsigned *dg_hist = nullptr;
    unsigned long long *dg_pref = nullptr, *dg_edges = nullptr;
    double *dg_acc = nullptr, *dg_tab = nullptr;
};

namespace {

int dev_alloc(pm_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail(PM_E_CUDA, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    c->allocs.push_back(*p);
    c->bytes += bytes;
    return PM_OK;
}

int tw_index(int L) {
    int i = 0;
    while ((16 << i) < L) ++i;
    return i;
}

template <typename T> PartK<T> part_k(const pm_particles *p) {
    PartK<T> k;
    k.x = (T *)p->x; k.y = (T *)p->y; k.z = (T *)p->z;
    k.vx = (T *)p->vx; k.vy = (T *)p->vy; k.vz = (T *)p->vz;
    k.m = (const T *)p->m;
    k.gal = p->gal;
    k.flags = p->flags;
    k.n = p->n;
    return k;
}

// After a synchronisation: a kernel's bounded wait that expired is reported.
int check_device_error(pm_ctx *c) {
    int h = 0;
    PM_CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    if (h == 2) return fail(PM_E_STATE, "an FFT pass was launched with a configuration it does not support");
    if (h) return fail(PM_E_TIMEOUT, "a tensor copy of an FFT pass did not complete within its time limit");
    return PM_OK;
}

int check_particles(const pm_particles *p) {
    if (!p) return fail(PM_E_ARG, "particles is NULL");
    if (p->n < 0) return fail(PM_E_ARG, "negative particle count %lld", (long long)p->n);
    if (p->n > 0 && (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->m || !p->gal || !p->flags))
        return fail(PM_E_ARG, "a particle array pointer is NULL");
    return PM_OK;
}

// --- H-hat: FP64 octant of H, three cosine sums, scaled into storage ---
int build_hhat(pm_ctx *c, GeoBuf &gb) {
    const pm_geometry &g = gb.g;
    const int P = g.nx + 1, Q = g.ny + 1, R = g.nz + 1;
    const long long n = (long long)P * Q * R;
    double *h = nullptr, *t1 = nullptr, *cm = nullptr;
    PM_CK(cudaMalloc(&h, n * sizeof(double)));
    PM_CK(cudaMalloc(&t1, n * sizeof(double)));
    const int nmax = std::max(P, std::max(Q, R));
    PM_CK(cudaMalloc(&cm, (size_t)nmax * nmax * sizeof(double)));
    std::vector<double> hm((size_t)nmax * nmax);
    auto cosmat = [&](int nn) {   // w_i cos(pi m i / nn), m, i in [0, nn]
        const int n1 = nn + 1;
        for (int m = 0; m < n1; ++m)
            for (int i = 0; i < n1; ++i) {
                const long long r = ((long long)m * i) % (2LL * nn);
                const double w = (i == 0 || i == nn) ? 1.0 : 2.0;
                hm[(size_t)m * n1 + i] = w * std::cos(M_PI * (double)r / (double)nn);
            }
        return cudaMemcpyAsync(cm, hm.data(), (size_t)n1 * n1 * sizeof(double), cudaMemcpyHostToDevice, c->user);
    };
    cudaStream_t st = c->user;
    PM_CK(pm_green_octant(h, g.nx, g.ny, g.nz, g.l_z / g.l_xy, c->sys.h000, st));
    PM_CK(cosmat(g.nx));
    PM_CK(pm_axis_transform(h, t1, cm, P, (long long)R * Q, 1, st));
    PM_CK(cudaStreamSynchronize(st));
    PM_CK(cosmat(g.ny));
    PM_CK(pm_axis_transform(t1, h, cm, Q, R, P, st));
    PM_CK(cudaStreamSynchronize(st));
    PM_CK(cosmat(g.nz));
    PM_CK(pm_axis_transform(h, t1, cm, R, 1, (long long)Q * P, st));
    const double scale = c->sys.G / (g.l_xy * 8.0 * g.nx * g.ny * g.nz);
    if (c->prec == PM_FP32) PM_CK(pm_store_hhat<float>(t1, (float *)gb.hhat, g.nx, g.ny, g.nz, scale, st));
    else PM_CK(pm_store_hhat<double>(t1, (double *)gb.hhat, g.nx, g.ny, g.nz, scale, st));
    PM_CK(cudaStreamSynchronize(st));
    cudaFree(h);
    cudaFree(t1);
    cudaFree(cm);
    return PM_OK;
}

template <typename T> int upload_twiddles(pm_ctx *c) {
    typedef typename cplx_t<T>::type C;
    for (int i = 0; i < 6; ++i) {
        const int L = 16 << i;
        std::vector<C> tw(L);
        for (int m = 0; m < L; ++m) {
            const double a = 2.0 * M_PI * (double)m / (double)L;
            tw[m].x = (T)std::cos(a);
            tw[m].y = (T)(-std::sin(a));
        }
        PM_TRY(dev_alloc(c, &c->d_tw[i], L * sizeof(C)));
        PM_CK(cudaMemcpyAsync(c->d_tw[i], tw.data(), L * sizeof(C), cudaMemcpyHostToDevice, c->user));
        PM_CK(cudaStreamSynchronize(c->user));
        // D(k) = exp(2 pi i k / L) - 1 = -2 sin^2(pi k / L) + i sin(2 pi k / L)
        // (the half-angle form keeps the real part accurate for small k)
        for (int m = 0; m < L; ++m) {
            const double h = std::sin(M_PI * (double)m / (double)L);
            tw[m].x = (T)(-2.0 * h * h);
            tw[m].y = (T)std::sin(2.0 * M_PI * (double)m / (double)L);
        }
        PM_TRY(dev_alloc(c, &c->d_dt[i], L * sizeof(C)));
        PM_CK(cudaMemcpyAsync(c->d_dt[i], tw.data(), L * sizeof(C), cudaMemcpyHostToDevice, c->user));
        PM_CK(cudaStreamSynchronize(c->user));
    }
    return PM_OK;
}

// ---- the passes of pm_solve --------------------------------------------------
enum { PASS_XFWD = 0, PASS_YFWD, PASS_ZCONV, PASS_YINV, PASS_XINV, NPASS };

// The arguments of one pair's passes.  shift: fixed-point scale of the
// input densities (2^-shift); the mass scale unless an adjoint solve passes
// its own.
PairArgs pair_args(const pm_ctx *c, const GeoBuf &gb, const Pair &pr, int shift) {
    const pm_geometry &g = gb.g;
    PairArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rho_a = c->rho[pr.gi][pr.a];
    a.rho_b = pr.b >= 0 ? c->rho[pr.gi][pr.b] : nullptr;
    a.work = pr.work;
    a.phi_b = pr.b >= 0 ? c->phi[pr.gi][pr.b] : nullptr;
    a.phi_sum = c->phi[pr.gi][pr.a];
    a.hhat = gb.hhat;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    a.scale = std::ldexp(1.0, -(shift == INT_MIN ? c->shift : shift));
    a.err = c->d_err;
    a.dtx = c->d_dt[tw_index(2 * g.nx)];
    a.dty = c->d_dt[tw_index(2 * g.ny)];
    a.dtz = c->d_dt[tw_index(2 * g.nz)];
    return a;
}

// Items of one batched pass launch (PairArgs and tensor maps).
struct BatchItems {
    std::vector<PairArgs> a;
    std::vector<const CUtensorMap *> l, s;
    void add(const PairArgs &x, const CUtensorMap *lm = nullptr, const CUtensorMap *sm = nullptr) {
        a.push_back(x);
        l.push_back(lm);
        s.push_back(sm ? sm : lm);
    }
};

// Launches `pass` of every item in chunks of `chunk` (<= PM_BATCH) items.
template <typename T> cudaError_t launch_items(int pass, const BatchItems &it, size_t chunk, cudaStream_t st) {
    for (size_t i0 = 0; i0 < it.a.size(); i0 += chunk) {
        PassBatch b;
        std::memset(&b, 0, sizeof(b));
        b.n = (int)std::min<size_t>(chunk, it.a.size() - i0);
        for (int k = 0; k < b.n; ++k) {
            b.a[k] = it.a[i0 + k];
            if (it.l[i0 + k]) b.lmap[k] = *it.l[i0 + k];
            if (it.s[i0 + k]) b.smap[k] = *it.s[i0 + k];
        }
        cudaError_t e;
        switch (pass) {
            case PASS_XFWD: e = pm_launch_xfwd<T>(b, st); break;
            case PASS_YFWD: e = pm_launch_col<T>(b, COL_YFWD, st); break;
            case PASS_ZCONV: e = pm_launch_col<T>(b, COL_ZCONV, st); break;
            case PASS_YINV: e = pm_launch_col<T>(b, COL_YINV, st); break;
            default: e = pm_launch_xinv<T>(b, st); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One pass of every pair of the units (only >= 0: of unit `only`); a
// unit's pairs share each pass's launches when the context batches (the
// pairs of a unit then have one shape).  A grid 1 pair (diff) takes part in
// the forward passes like any other; its z pass forms H-hat (D_x + i D_y)
// into work2 and H-hat (D_z + i) in place, in one launch from one forward
// transform (dmode 3: z lengths up to 64, and 128 and 256 where a tile's
// columns fit in nx) or else in two launches (dmode 1, then 2); its inverse
// passes run on both work arrays: fx + i fy -> fx, fy; fz + i Phi_1 -> fz,
// Phi_1.
template <typename T> int launch_pass(pm_ctx *c, int pass, cudaStream_t st, int only = -1, int shift = INT_MIN) {
    const size_t chunk = c->batched ? PM_BATCH : 1;
    for (int ui = 0; ui < (int)c->units.size(); ++ui) {
        if (only >= 0 && ui != only) continue;
        BatchItems main, d1, d2;
        for (int gi : c->units[ui]) {
            const GeoBuf &gb = c->geos[gi];
            const pm_geometry &sg = gb.g;
            for (const Pair &pr : gb.pairs) {
                PairArgs a = pair_args(c, gb, pr, shift);
                switch (pass) {
                    case PASS_XFWD:
                        a.tw = c->d_tw[tw_index(2 * sg.nx)];
                        main.add(a);
                        break;
                    case PASS_YFWD:
                        a.tw = c->d_tw[tw_index(2 * sg.ny)];
                        main.add(a, &pr.yfwd, &pr.yinv);   // stores: boxes of 2ny rows
                        break;
                    case PASS_ZCONV:
                        a.tw = c->d_tw[tw_index(2 * sg.nz)];
                        if (!pr.diff) {
                            main.add(a, &pr.zmap);
                        } else if (sg.nz <= 32 ||
                                   ((sg.nz == 64 || sg.nz == 128) && pm_col_cols(2 * sg.nz, (int)c->esz) <= sg.nx)) {
                            // both difference fields from one forward transform (H-hat read from the
                            // thread-major table, L <= 64, or from the tile's staged rows)
                            a.dmode = 3;
                            d1.add(a, &pr.zmap, &pr.zmap2);
                        } else {
                            a.dmode = 1;
                            d1.add(a, &pr.zmap, &pr.zmap2);
                            a.dmode = 2;
                            d2.add(a, &pr.zmap);
                        }
                        break;
                    case PASS_YINV:
                        a.tw = c->d_tw[tw_index(2 * sg.ny)];
                        main.add(a, &pr.yinv, &pr.yfwd);   // stores: boxes of ny rows
                        if (pr.diff) {
                            a.work = pr.work2;
                            main.add(a, &pr.yinv2, &pr.yfwd2);
                        }
                        break;
                    default:
                        a.tw = c->d_tw[tw_index(2 * sg.nx)];
                        if (pr.diff) {
                            a.split = 1;
                            a.phi_sum = c->fd[pr.gi][2];
                            a.phi_b = c->phi[pr.gi][pr.a];
                            main.add(a);
                            a.work = pr.work2;
                            a.phi_sum = c->fd[pr.gi][0];
                            a.phi_b = c->fd[pr.gi][1];
                        }
                        main.add(a);
                        break;
                }
            }
        }
        cudaError_t e = launch_items<T>(pass, main, chunk, st);
        if (e == cudaSuccess) e = launch_items<T>(pass, d1, chunk, st);
        if (e == cudaSuccess) e = launch_items<T>(pass, d2, chunk, st);
        if (e != cudaSuccess) return fail(PM_E_CUDA, "FFT pass %d launch failed: %s", pass, cudaGetErrorString(e));
    }
    return PM_OK;
}

// With ev (phase timing) the passes run pass by pass on st.  Otherwise the
// units' chains of five passes run on branch streams forked from and joined
// back to st, by one of two schedules (timed at creation with and without
// batching, the fastest kept): one branch per unit, all chains starting
// together; or two lanes of about equal work, one taking its chains largest
// first and the other smallest first, so that the compute-bound z pass of
// one large chain meets the bandwidth-bound x and y passes of another rather
// than its own z pass.
template <typename T> int enqueue_solve(pm_ctx *c, cudaStream_t st, cudaEvent_t *ev, int shift = INT_MIN) {
    if (ev || c->units.size() < 2) {
        for (int pass = 0; pass < NPASS; ++pass) {
            PM_TRY(launch_pass<T>(c, pass, st, -1, shift));
            if (ev) PM_CK(cudaEventRecord(ev[pass], st));
        }
        return PM_OK;
    }
    PM_CK(cudaEventRecord(c->ev_fork, st));
    if (c->sched == 0) {
        for (int gi = 0; gi < (int)c->units.size(); ++gi) {
            cudaStream_t b = c->branch[gi];
            PM_CK(cudaStreamWaitEvent(b, c->ev_fork, 0));
            for (int pass = 0; pass < NPASS; ++pass) PM_TRY(launch_pass<T>(c, pass, b, gi, shift));
            PM_CK(cudaEventRecord(c->ev_join[gi], b));
            PM_CK(cudaStreamWaitEvent(st, c->ev_join[gi], 0));
        }
        return PM_OK;
    }
    for (size_t l = 0; l < c->lanes.size(); ++l) {
        cudaStream_t b = c->branch[l];
        PM_CK(cudaStreamWaitEvent(b, c->ev_fork, 0));
        for (int gi : c->lanes[l])
            for (int pass = 0; pass < NPASS; ++pass) PM_TRY(launch_pass<T>(c, pass, b, gi, shift));
        PM_CK(cudaEventRecord(c->ev_join[l], b));
        PM_CK(cudaStreamWaitEvent(st, c->ev_join[l], 0));
    }
    return PM_OK;
}

// Two lanes of about equal transform volume: the units' chains taken
// largest first, the first to lane 0, each next one to the lighter lane
// (lane 1 on ties); lane 0 runs largest first, lane 1 smallest first, so
// lane 1's large chains start after its small ones.
std::vector<std::vector<int>> plan_lanes(const std::vector<std::vector<int>> &units, const std::vector<GeoBuf> &geos) {
    std::vector<std::pair<double, int>> w;
    for (int ui = 0; ui < (int)units.size(); ++ui) {
        double vol = 0;
        for (int gi : units[ui]) {
            const pm_geometry &g = geos[gi].g;
            vol += 8.0 * g.nx * g.ny * g.nz * (double)geos[gi].pairs.size();
        }
        w.push_back({vol, ui});
    }
    std::sort(w.begin(), w.end(), [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
        return a.first != b.first ? a.first > b.first : a.second < b.second;
    });
    std::vector<std::vector<int>> lanes(2);
    double tot[2] = {0, 0};
    for (const auto &x : w) {
        const int l = lanes[0].empty() ? 0 : (tot[0] < tot[1] ? 0 : 1);
        lanes[l].push_back(x.second);
        tot[l] += x.first;
    }
    std::reverse(lanes[1].begin(), lanes[1].end());
    if (lanes[1].empty()) lanes.pop_back();
    return lanes;
}

// Units of the solve: shapes (batched) or single geometries.
void set_units(pm_ctx *c, bool batched) {
    c->batched = batched;
    c->units.clear();
    if (batched) {
        for (const ShapeGroup &sg : c->shapes) c->units.push_back(sg.geos);
    } else {
        for (int gi = 0; gi < (int)c->geos.size(); ++gi) c->units.push_back({gi});
    }
    c->lanes = plan_lanes(c->units, c->geos);
}

// Chooses the solve's launch configuration by timing: batched or per-pair
// launches, and the two branch schedules.  Every configuration is timed
// (four solves after one untimed) in three interleaved rounds and keeps its
// fastest round, so that a transient slowdown does not decide the choice.
template <typename T> int tune_schedule(pm_ctx *c) {
    set_units(c, true);
    c->sched = 0;
    if (c->geos.size() < 2) return PM_OK;
    PM_CK(cudaMemsetAsync(c->rho_all, 0, c->rho_bytes, c->user));
    cudaEvent_t e0, e1;
    PM_CK(cudaEventCreate(&e0));
    PM_CK(cudaEventCreate(&e1));
    struct Cfg { int bt, sc; float ms; };
    std::vector<Cfg> cfg;
    for (int bt = 1; bt >= 0; --bt) {
        set_units(c, bt != 0);
        for (int sc = 0; sc < (c->units.size() < 2 ? 1 : 2); ++sc) cfg.push_back({bt, sc, -1.f});
    }
    int rc = PM_OK;
    for (int round = 0; round < 3 && rc == PM_OK; ++round)
        for (Cfg &f : cfg) {
            if (rc != PM_OK) break;
            set_units(c, f.bt != 0);
            c->sched = f.sc;
            rc = enqueue_solve<T>(c, c->user, nullptr);
            if (rc == PM_OK && cudaEventRecord(e0, c->user) != cudaSuccess) rc = fail(PM_E_CUDA, "event record failed");
            for (int k = 0; k < 4 && rc == PM_OK; ++k) rc = enqueue_solve<T>(c, c->user, nullptr);
            if (rc == PM_OK && cudaEventRecord(e1, c->user) != cudaSuccess) rc = fail(PM_E_CUDA, "event record failed");
            float ms = 0.f;
            if (rc == PM_OK &&
                (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = fail(PM_E_CUDA, "schedule timing failed");
            if (rc == PM_OK && (f.ms < 0.f || ms < f.ms)) f.ms = ms;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const Cfg *best = &cfg[0];
    for (const Cfg &f : cfg)
        if (f.ms >= 0.f && (best->ms < 0.f || f.ms < best->ms)) best = &f;
    set_units(c, best->bt != 0);
    c->sched = best->sc;
    if (rc != PM_OK) return rc;
    return check_device_error(c);
}

template <typename T> int enqueue_deposit(pm_ctx *c, const pm_particles *p, cudaStream_t st) {
    PM_CK(cudaMemsetAsync(c->rho_all, 0, c->rho_bytes, st));
    PM_CK(pm_launch_deposit<T>(part_k<T>(p), c->hs, c->d_cen, c->sort_interval > 0 ? 1 : 0, st));
    return PM_OK;
}

// phase: 3 = sums and apply, 1 = sums only, 2 = apply only (a sharded step
// sums each rank's particles, adds the accumulators across ranks, applies).
template <typename T> int enqueue_recentre(pm_ctx *c, const pm_particles *p, cudaStream_t st, int phase = 3) {
    if (!c->any_recentre) return PM_OK;
    PM_CK(pm_launch_recentre<T>(part_k<T>(p), c->hs, c->d_cen, c->d_csum, phase, st));
    return PM_OK;
}

// One full step; ev (optional, 8 events) marks the phase boundaries.
template <typename T> int enqueue_step(pm_ctx *c, const pm_particles *p, double dt, cudaStream_t st,
                                       cudaEvent_t *ev) {
    PM_TRY(enqueue_recentre<T>(c, p, st));
    if (ev) PM_CK(cudaEventRecord(ev[0], st));
    PM_TRY(enqueue_deposit<T>(c, p, st));
    if (ev) PM_CK(cudaEventRecord(ev[1], st));
    PM_TRY(enqueue_solve<T>(c, st, ev ? ev + 2 : nullptr));
    PM_CK(pm_launch_force<T>(0, part_k<T>(p), c->hs, c->d_cen, dt, nullptr, nullptr, nullptr, nullptr, st));
    if (ev) PM_CK(cudaEventRecord(ev[7], st));
    return PM_OK;
}

void destroy_set(GraphSet &g) {
    for (int k = 0; k < 2; ++k) {
        if (g.gexec[k]) cudaGraphExecDestroy(g.gexec[k]);
        if (g.graph[k]) cudaGraphDestroy(g.graph[k]);
        g.gexec[k] = nullptr;
        g.graph[k] = nullptr;
    }
    g.valid = false;
}

void destroy_graph(pm_ctx *c) {
    for (GraphSet &g : c->gs) destroy_set(g);
}

// Scratch of the spatial sort for n particles (allocated outside any capture).
int ensure_sort_scratch(pm_ctx *c, long long n) {
    if (n <= c->sort_cap) return PM_OK;
    destroy_graph(c);   // captured steps hold the old scratch's addresses
    for (int k = 0; k < 9; ++k)
        PM_TRY(dev_alloc(c, &c->s_arr[k], (size_t)n * (k < 7 ? c->esz : 4)));
    PM_TRY(dev_alloc(c, (void **)&c->s_key, (size_t)n * 4));
    PM_TRY(dev_alloc(c, (void **)&c->s_rank, (size_t)n * 4));
    c->sort_cap = n;
    return PM_OK;
}

template <typename T> int enqueue_sort(pm_ctx *c, const pm_particles *p, long long *perm, cudaStream_t st) {
    PartK<T> scratch = part_k<T>(p);
    scratch.x = (T *)c->s_arr[0]; scratch.y = (T *)c->s_arr[1]; scratch.z = (T *)c->s_arr[2];
    scratch.vx = (T *)c->s_arr[3]; scratch.vy = (T *)c->s_arr[4]; scratch.vz = (T *)c->s_arr[5];
    scratch.m = (const T *)c->s_arr[6];
    scratch.gal = (const int32_t *)c->s_arr[7];
    scratch.flags = (uint32_t *)c->s_arr[8];
    PM_CK(pm_launch_sort<T>(part_k<T>(p), scratch, c->hs, c->d_cen, c->sortk, c->s_count, c->s_key,
                            c->s_rank, c->s_bsum, perm, st));
    return PM_OK;
}

template <typename T> int capture(pm_ctx *c, const pm_particles *p, double dt, bool with_sort,
                                  cudaGraph_t *gr, cudaGraphExec_t *ex) {
    PM_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int rc = with_sort ? enqueue_sort<T>(c, p, nullptr, c->cap) : PM_OK;
    if (rc == PM_OK) rc = enqueue_step<T>(c, p, dt, c->cap, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (rc != PM_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(PM_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    *gr = g;
    e = cudaGraphInstantiate(ex, g, 0);
    if (e != cudaSuccess) return fail(PM_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    return PM_OK;
}

template <typename T> int step_impl(pm_ctx *c, const pm_particles *p, double dt, int nsteps) {
    const bool sorting = c->sort_interval > 0 && p->n > 0;
    GraphSet *gs = nullptr;
    for (GraphSet &g : c->gs)
        if (g.valid && std::memcmp(&g.key, p, sizeof(pm_particles)) == 0 && g.dt == dt) gs = &g;
    if (!gs) {
        if (sorting) PM_TRY(ensure_sort_scratch(c, p->n));
        for (GraphSet &g : c->gs) {
            if (!g.valid) { gs = &g; break; }
            if (!gs || g.used < gs->used) gs = &g;
        }
        destroy_set(*gs);
        std::memcpy(&gs->key, p, sizeof(pm_particles));
        gs->dt = dt;
        gs->valid = true;
    }
    gs->used = ++c->guse;
    for (int s = 0; s < nsteps; ++s) {
        const bool sort_now = sorting && c->step_count % c->sort_interval == 0;
        const int g = sort_now ? 1 : 0;
        if (!gs->gexec[g]) {
            const int rc = capture<T>(c, p, dt, sort_now, &gs->graph[g], &gs->gexec[g]);
            if (rc != PM_OK) { destroy_set(*gs); return rc; }
        }
        PM_CK(cudaGraphLaunch(gs->gexec[g], c->user));
        ++c->step_count;
    }
    return PM_OK;
}

template <typename T> int step_timed_impl(pm_ctx *c, const pm_particles *p, double dt, int nsteps, float *ms) {
    const int NE = 10;
    const bool sorting = c->sort_interval > 0 && p->n > 0;
    if (sorting) PM_TRY(ensure_sort_scratch(c, p->n));
    std::vector<cudaEvent_t> ev((size_t)nsteps * NE);
    for (auto &e : ev) PM_CK(cudaEventCreate(&e));
    int rc = PM_OK;
    for (int s = 0; s < nsteps && rc == PM_OK; ++s) {
        cudaEvent_t *e = ev.data() + (size_t)s * NE;
        cudaEventRecord(e[9], c->user);
        if (sorting && c->step_count % c->sort_interval == 0) rc = enqueue_sort<T>(c, p, nullptr, c->user);
        ++c->step_count;
        cudaEventRecord(e[0], c->user);
        if (rc == PM_OK) rc = enqueue_step<T>(c, p, dt, c->user, e + 1);
    }
    for (int k = 0; k < 10; ++k) ms[k] = 0.f;
    if (rc == PM_OK) {
        cudaError_t er = cudaStreamSynchronize(c->user);
        if (er != cudaSuccess) rc = fail(PM_E_CUDA, "step_timed sync: %s", cudaGetErrorString(er));
    }
    if (rc == PM_OK) {
        for (int s = 0; s < nsteps; ++s) {
            cudaEvent_t *e = ev.data() + (size_t)s * NE;
            for (int k = 0; k < 8; ++k) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e[k], e[k + 1]);
                ms[k] += t;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e[9], e[8]);
            ms[8] += t;
            cudaEventElapsedTime(&t, e[9], e[0]);
            ms[9] += t;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    return rc;
}

// ---- CIC variant (differentiable runs) -------------------------------------
template <typename T> int cic_deposit_impl(pm_ctx *c, const pm_particles *p) {
    PM_CK(cudaMemsetAsync(c->rho_all, 0, c->rho_bytes, c->user));
    PM_CK(pm_launch_cic_deposit<T>(part_k<T>(p), c->hs, c->d_cen, c->user));
    return PM_OK;
}

template <typename T> int cic_field_impl(pm_ctx *c, int mode, const pm_particles *p, double dtk, double dtd,
                                         void *ox, void *oy, void *oz) {
    PM_CK(pm_launch_cic_field<T>(mode, part_k<T>(p), c->hs, c->d_cen, dtk, dtd, (T *)ox, (T *)oy, (T *)oz, nullptr,
                                 nullptr, nullptr, 0.0, c->user));
    return PM_OK;
}

// Largest (2 c_gx + c_gz) = 1/l_xy + 1/(2 l_z) over the grids: bounds one
// particle's adjoint density in any cell per unit |u|.
double cic_coef_bound(const SysK &hs) {
    double b = 0;
    for (int g = 0; g < hs.ngal; ++g) {
        const GeomK *gs[3] = {&hs.gal[g].fine, &hs.gal[g].med, &hs.gal[g].coarse};
        for (const GeomK *k : gs)
            if (k->nx) b = std::max(b, 2.0 * k->c_gx + k->c_gz);
    }
    return b;
}

template <typename T> int cic_vjp_impl(pm_ctx *c, const pm_particles *p, const void *ux, const void *uy,
                                       const void *uz, void *gx, void *gy, void *gz, void *gm) {
    const PartK<T> pk = part_k<T>(p);
    const T *u[3] = {(const T *)ux, (const T *)uy, (const T *)uz};
    // direct term, with the forward potentials still in place
    PM_CK(pm_launch_cic_field<T>(2, pk, c->hs, c->d_cen, 0.0, 0.0, (T *)gx, (T *)gy, (T *)gz, u[0], u[1], u[2], 0.0,
                                 c->user));
    // fixed-point scale of the adjoint densities: |cell sum| <= n max|u| bound
    PM_CK(cudaMemsetAsync(c->d_cnt, 0, sizeof(unsigned long long), c->user));
    PM_CK(pm_launch_cic_umax<T>(pk, u[0], u[1], u[2], (unsigned *)c->d_cnt, c->user));
    unsigned bits = 0;
    PM_CK(cudaMemcpyAsync(&bits, c->d_cnt, sizeof(bits), cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    float umax;
    std::memcpy(&umax, &bits, sizeof(umax));
    if (!std::isfinite(umax)) return fail(PM_E_ARG, "cotangent has a non-finite entry");
    if (umax == 0.f) return check_device_error(c);
    const double bound = 1.01 * (double)p->n * (double)umax * cic_coef_bound(c->hs);
    int sa = 61 - ceil_log2(bound);
    sa = std::min(120, std::max(-100, sa));
    PM_CK(cudaMemsetAsync(c->rho_all, 0, c->rho_bytes, c->user));
    PM_CK(pm_launch_cic_field<T>(3, pk, c->hs, c->d_cen, 0.0, 0.0, nullptr, nullptr, nullptr, u[0], u[1], u[2],
                                 std::ldexp(1.0, sa), c->user));
    PM_TRY(enqueue_solve<T>(c, c->user, nullptr, sa));
    PM_CK(pm_launch_cic_gather<T>(pk, c->hs, c->d_cen, (T *)gx, (T *)gy, (T *)gz, (T *)gm, c->user));
    return check_device_error(c);
}

// ---- disc diagnostics (Sec. 6 quantities) ----------------------------------
constexpr int DG_MAXBINS = 64, DG_MAXRM = 1024;

template <typename T> int disc_impl(pm_ctx *c, const pm_particles *p, const uint8_t *sel, const pm_disc_query *q,
                                    double *out) {
    cudaStream_t st = c->user;
    if (!c->dg_hist) {
        PM_TRY(dev_alloc(c, (void **)&c->dg_hist, sizeof(unsigned) * 256 * DG_MAXBINS));
        PM_TRY(dev_alloc(c, (void **)&c->dg_pref, sizeof(unsigned long long) * DG_MAXBINS));
        PM_TRY(dev_alloc(c, (void **)&c->dg_edges, sizeof(unsigned long long) * DG_MAXBINS));
        PM_TRY(dev_alloc(c, (void **)&c->dg_acc, sizeof(double) * (4 * DG_MAXBINS + 8 + 2 * DG_MAXRM)));
        PM_TRY(dev_alloc(c, (void **)&c->dg_tab, sizeof(double) * 2 * DG_MAXBINS));
    }
    CenK ck;
    PM_CK(cudaMemcpyAsync(&ck, c->d_cen, sizeof(CenK), cudaMemcpyDeviceToHost, st));
    PM_CK(cudaStreamSynchronize(st));
    pmk::DiagP<T> d;
    d.x = (const T *)p->x; d.y = (const T *)p->y; d.z = (const T *)p->z;
    d.vx = (const T *)p->vx; d.vy = (const T *)p->vy; d.vz = (const T *)p->vz;
    d.m = (const T *)p->m;
    d.flags = p->flags;
    d.sel = sel;
    d.gal_id = p->gal;
    d.gal = q->gal;
    d.n = p->n;
    for (int k = 0; k < 3; ++k) d.c[k] = ck.c[q->gal][k];
    const int B = q->nbins, NR = q->nring, MM = q->mmax;
    const int nacc = 4 * B + 7 + 2 * NR * MM;
    const int nout = 6 + 4 * B + 2 * NR * MM;
    for (int k = 0; k < nout; ++k) out[k] = 0.0;

    // exact bin edges: order statistics of R^2 at ranks floor(k n / B)
    std::vector<unsigned long long> key(B > 1 ? B - 1 : 0, 0ull);
    std::vector<long long> rank(key.size(), 0);
    long long nsel = -1;
    std::vector<unsigned> h(256 * DG_MAXBINS);
    for (int pass = 0; pass < 8 && (!key.empty()); ++pass) {
        std::vector<unsigned long long> uniq(key.begin(), key.end());
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        const int np = pass == 0 ? 1 : (int)uniq.size();
        PM_CK(cudaMemcpyAsync(c->dg_pref, uniq.data(), sizeof(unsigned long long) * np, cudaMemcpyHostToDevice, st));
        PM_CK(cudaMemsetAsync(c->dg_hist, 0, sizeof(unsigned) * 256 * np, st));
        PM_CK(pm_launch_diag_hist<T>(d, pass, c->dg_pref, np, c->dg_hist, st));
        PM_CK(cudaMemcpyAsync(h.data(), c->dg_hist, sizeof(unsigned) * 256 * np, cudaMemcpyDeviceToHost, st));
        PM_CK(cudaStreamSynchronize(st));
        if (pass == 0) {
            nsel = 0;
            for (int b = 0; b < 256; ++b) nsel += h[b];
            if (nsel == 0) return check_device_error(c);
            for (int k = 1; k < B; ++k) rank[k - 1] = ((long long)k * nsel) / B;
        }
        for (size_t k = 0; k < key.size(); ++k) {
            const int j = pass == 0 ? 0 : (int)(std::lower_bound(uniq.begin(), uniq.end(), key[k]) - uniq.begin());
            long long cum = 0;
            int dgt = 0;
            for (; dgt < 256; ++dgt) {
                if (cum + h[j * 256 + dgt] > rank[k]) break;
                cum += h[j * 256 + dgt];
            }
            if (dgt == 256) return fail(PM_E_STATE, "radix select lost a rank (particles changed during the call?)");
            key[k] = (key[k] << 8) | (unsigned long long)dgt;
            rank[k] -= cum;
        }
    }
    if (!key.empty())
        PM_CK(cudaMemcpyAsync(c->dg_edges, key.data(), sizeof(unsigned long long) * key.size(), cudaMemcpyHostToDevice,
                              st));
    pmk::DiagQ dq;
    dq.nbins = B; dq.nring = NR; dq.mmax = MM;
    dq.r_ring = q->r_ring;
    dq.width = NR > 0 ? q->r_ring / NR : 1.0;
    dq.rlo = q->r0 - q->dr;
    dq.rhi = q->r0 + q->dr;
    PM_CK(cudaMemsetAsync(c->dg_acc, 0, sizeof(double) * (nacc + 1), st));
    PM_CK(pm_launch_diag_sums<T>(d, dq, c->dg_edges, c->dg_acc, st));
    std::vector<double> acc(nacc + 1);
    PM_CK(cudaMemcpyAsync(acc.data(), c->dg_acc, sizeof(double) * nacc, cudaMemcpyDeviceToHost, st));
    PM_CK(cudaStreamSynchronize(st));

    std::vector<double> xp, fp;
    long long ntot = 0;
    for (int b = 0; b < B; ++b) {
        const double cnt = acc[4 * b + 1];
        ntot += (long long)cnt;
        double *o = out + 6 + 4 * b;
        o[1] = cnt;
        if (cnt > 0) {
            o[0] = acc[4 * b] / cnt;
            o[2] = std::sqrt(acc[4 * b + 2] / cnt);
            o[3] = acc[4 * b + 3] / cnt;
            xp.push_back(o[0]);
            fp.push_back(o[3]);
        }
    }
    out[0] = (double)ntot;
    const double *a = acc.data() + 4 * B;
    out[5] = a[0];
    if (a[0] > 0) {
        auto disp = [&](int k) {
            const double mean = a[k] / a[0];
            return std::sqrt(std::max(a[k + 1] / a[0] - mean * mean, 0.0));
        };
        out[2] = disp(1);
        out[3] = disp(3);
        out[4] = disp(5);
    }
    for (int r = 0; r < NR; ++r) {
        const double S = M_PI * (((r + 1) * dq.width) * ((r + 1) * dq.width) - (r * dq.width) * (r * dq.width));
        for (int mo = 0; mo < MM; ++mo)
            for (int k = 0; k < 2; ++k) out[6 + 4 * B + 2 * (r * MM + mo) + k] = a[7 + 2 * (r * MM + mo) + k] / S;
    }
    if (!xp.empty()) {
        std::vector<double> tab(xp);
        tab.insert(tab.end(), fp.begin(), fp.end());
        PM_CK(cudaMemcpyAsync(c->dg_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st));
        PM_CK(cudaMemsetAsync(c->dg_acc + nacc, 0, sizeof(double), st));
        PM_CK(pm_launch_diag_heat<T>(d, c->dg_tab, c->dg_tab + xp.size(), (int)xp.size(), c->dg_acc + nacc, st));
        PM_CK(cudaMemcpyAsync(&out[1], c->dg_acc + nacc, sizeof(double), cudaMemcpyDeviceToHost, st));
        PM_CK(cudaStreamSynchronize(st));
    }
    return check_device_error(c);
}

template <typename T> int force_impl(pm_ctx *c, int mode, const pm_particles *p, double dt, void *ax, void *ay,
                                     void *az, double *diag) {
    PM_CK(pm_launch_force<T>(mode, part_k<T>(p), c->hs, c->d_cen, dt, (T *)ax, (T *)ay, (T *)az, diag, c->user));
    return PM_OK;
}

}  // namespace

// ---- tensor maps of the column passes --------------------------------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2D map over 8-byte elements: dim0 contiguous, dim1 rows of stride1 bytes.
int encode2d(CUtensorMap *m, void *base, unsigned long long dim0, unsigned long long dim1,
             unsigned long long stride1, unsigned box0, unsigned box1,
             CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE) {
    EncodeTiledFn f = encode_fn();
    if (!f) return fail(PM_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t gdim[2] = {dim0, dim1};
    const cuuint64_t gstr[1] = {stride1};
    const cuuint32_t box[2] = {box0, box1};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PM_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PM_OK;
}
}  // namespace

int pm_encode_col_maps(void *work, int nx, int ny, int nz, int esz, CUtensorMap *yfwd, CUtensorMap *yinv,
                       CUtensorMap *zmap) {
    const unsigned long long epc = esz == 4 ? 1 : 2;   // 8-byte elements per complex value
    const unsigned long long nx2 = 2ull * nx, ny2 = 2ull * ny;
    const unsigned cy = (unsigned)pm_col_cols(2 * ny, esz), sz = (unsigned)pm_zsub_cols(2 * nz, esz);
    const unsigned zrow = sz * (unsigned)epc * 8;   // bytes per z box row: 32, 64 or 128
    const CUtensorMapSwizzle zswz = zrow >= 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                    : zrow >= 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                    : zrow >= 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE;
    // y passes: dim0 = kx, dim1 = the (z, y) rows, box = COLS columns x rows
    PM_TRY(encode2d(yfwd, work, nx2 * epc, ny2 * nz, nx2 * epc * 8, cy * (unsigned)epc, (unsigned)std::min(ny, 256)));
    PM_TRY(encode2d(yinv, work, nx2 * epc, ny2 * nz, nx2 * epc * 8, cy * (unsigned)epc,
                    (unsigned)std::min(2 * ny, 256)));
    // z pass: dim0 = the (ky, kx) columns, dim1 = z
    PM_TRY(encode2d(zmap, work, nx2 * ny2 * epc, nz, nx2 * ny2 * epc * 8, sz * (unsigned)epc,
                    (unsigned)std::min(nz, 256), zswz));
    return PM_OK;
}

PassBatch pm_single_batch(const PairArgs &a, const CUtensorMap *lmap, const CUtensorMap *smap) {
    PassBatch b;
    std::memset(&b, 0, sizeof(b));
    b.n = 1;
    b.a[0] = a;
    if (lmap) b.lmap[0] = *lmap;
    if (smap || lmap) b.smap[0] = smap ? *smap : *lmap;
    return b;
}

int pm_internal_fail(int code, const char *msg) {
    g_err = msg;
    return code;
}

// ============================================================================
extern "C" {

double pm_cell_length(double R, int32_t N, double q) { return 2.0 * R * q / (double)(N - 4); }

double pm_q_crit(double r_core, double r_out, double r_sys, int32_t N) {
    return std::fmax(r_core / r_out, 4.0 / (double)(N - 4) * r_sys / r_out);
}

int32_t pm_fixed_shift(double mass_bound) {
    if (!(mass_bound > 0) || !std::isfinite(mass_bound)) return INT32_MIN;
    return 62 - ceil_log2(mass_bound);
}

const char *pm_last_error(void) { return g_err.c_str(); }

int pm_create_grids(const pm_system *sys, const pm_galaxy *gals, void *stream, pm_ctx **out) {
    if (!out) return fail(PM_E_ARG, "out is NULL");
    *out = nullptr;
    if (!sys || !gals) return fail(PM_E_ARG, "sys or gals is NULL");
    if (sys->precision != PM_FP32 && sys->precision != PM_FP64)
        return fail(PM_E_ARG, "precision must be PM_FP32 or PM_FP64");
    if (sys->ngal < 1 || sys->ngal > PM_MAX_GALAXIES) return fail(PM_E_ARG, "ngal %d out of range", sys->ngal);
    if (!(sys->mass_bound > 0) || !std::isfinite(sys->mass_bound)) return fail(PM_E_ARG, "mass_bound must be positive and finite");
    if (!std::isfinite(sys->G) || !std::isfinite(sys->h000) || !(sys->r_sys > 0) || !std::isfinite(sys->r_sys))
        return fail(PM_E_ARG, "G, h000 must be finite and r_sys positive");
    const int shift = 62 - ceil_log2(sys->mass_bound);
    if (shift < -60 || shift > 1000) return fail(PM_E_OVERFLOW, "mass_bound %g leaves no fixed-point range", sys->mass_bound);

    for (int gi = 0; gi < sys->ngal; ++gi) {
        const pm_galaxy &G = gals[gi];
        if (!geom_present(G.coarse) || !geom_valid(G.coarse))
            return fail(PM_E_ARG, "galaxy %d: coarse grid must be present, powers of two in [8,256], positive lengths", gi);
        if (geom_present(G.fine) && !geom_present(G.medium))
            return fail(PM_E_ARG, "galaxy %d: a fine grid needs a medium grid", gi);
        if (geom_present(G.medium)) {
            if (!geom_valid(G.medium)) return fail(PM_E_ARG, "galaxy %d: invalid medium grid", gi);
            if (!(G.r_out > 0) || !(G.r_core >= 0) || G.r_core > G.r_out)
                return fail(PM_E_NESTING, "galaxy %d: need 0 <= r_core <= r_out, r_out > 0", gi);
            const double q = G.medium.l_z / G.medium.l_xy;
            if (q < 1.0) {
                if (gi != 0) return fail(PM_E_QCRIT, "galaxy %d: only the first galaxy may be flattened", gi);
                const double qc = pm_q_crit(G.r_core, G.r_out, sys->r_sys, G.medium.nx);
                if (q < qc * (1.0 - 1e-12)) return fail(PM_E_QCRIT, "galaxy %d: q = %g below q_crit = %g", gi, q, qc);
            }
            if (ext_xy(G.medium, G.medium.nx) > ext_xy(G.coarse, G.coarse.nx) ||
                ext_xy(G.medium, G.medium.ny) > ext_xy(G.coarse, G.coarse.ny) || ext_z(G.medium) > ext_z(G.coarse))
                return fail(PM_E_NESTING, "galaxy %d: medium grid larger than coarse grid", gi);
        }
        if (geom_present(G.fine)) {
            if (!geom_valid(G.fine)) return fail(PM_E_ARG, "galaxy %d: invalid fine grid", gi);
            if (ext_xy(G.fine, G.fine.nx) > ext_xy(G.medium, G.medium.nx) ||
                ext_xy(G.fine, G.fine.ny) > ext_xy(G.medium, G.medium.ny) || ext_z(G.fine) > ext_z(G.medium))
                return fail(PM_E_NESTING, "galaxy %d: fine grid larger than medium grid", gi);
        }
        if (G.recentre && !(G.r_core > 0)) return fail(PM_E_ARG, "galaxy %d: recentring needs r_core > 0", gi);
    }

    pm_ctx *c = new pm_ctx();
    c->sys = *sys;
    for (int gi = 0; gi < sys->ngal; ++gi) c->gal[gi] = gals[gi];
    c->prec = sys->precision;
    c->esz = sys->precision == PM_FP32 ? 4 : 8;
    c->shift = shift;
    c->mscale = std::ldexp(1.0, shift);
    c->user = (cudaStream_t)stream;
    std::memset(c->set_geo, -1, sizeof(c->set_geo));
    std::memset(c->rho, 0, sizeof(c->rho));
    std::memset(c->phi, 0, sizeof(c->phi));
    std::memset(c->fd, 0, sizeof(c->fd));

    auto cleanup = [&](int rc) { pm_destroy(c); return rc; };
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return cleanup(fail(PM_E_CUDA, "cudaStreamCreate failed"));
    cudaError_t ea = (c->prec == PM_FP32) ? pm_set_attrs<float>() : pm_set_attrs<double>();
    if (ea != cudaSuccess) return cleanup(fail(PM_E_CUDA, "kernel attributes: %s", cudaGetErrorString(ea)));

    // geometries and mass sets
    auto add_set = [&](int gi, int k, const pm_geometry &g) {
        int id = -1;
        for (size_t i = 0; i < c->geos.size(); ++i)
            if (geom_equal(c->geos[i].g, g)) id = (int)i;
        if (id < 0) {
            GeoBuf gb;
            gb.g = g;
            gb.A = (long long)g.nx * g.ny * g.nz;
            gb.workN = (long long)g.nz * 2 * g.ny * 2 * g.nx;
            gb.hatN = pm_hhat_table_size(g.nx, g.ny, g.nz);
            c->geos.push_back(gb);
            id = (int)c->geos.size() - 1;
        }
        c->geos[id].sets.push_back({gi, k});
        c->set_geo[gi][k] = id;
    };
    for (int gi = 0; gi < sys->ngal; ++gi) {
        const pm_galaxy &G = gals[gi];
        if (geom_present(G.fine)) add_set(gi, 0, G.fine);
        if (geom_present(G.medium)) {
            add_set(gi, 1, G.medium);
            add_set(gi, 2, G.medium);
            add_set(gi, 3, G.coarse);
        }
        add_set(gi, 4, G.coarse);
        if (G.recentre) c->any_recentre = true;
    }
    size_t rho_total = 0;
    for (int gi = 0; gi < sys->ngal; ++gi)
        for (int k = 0; k < PM_SETS; ++k)
            if (c->set_geo[gi][k] >= 0) rho_total += (size_t)c->geos[c->set_geo[gi][k]].A;
    int rc;
    if ((rc = dev_alloc(c, (void **)&c->rho_all, rho_total * 8))) return cleanup(rc);
    c->rho_bytes = rho_total * 8;
    size_t off = 0;
    for (int gi = 0; gi < sys->ngal; ++gi)
        for (int k = 0; k < PM_SETS; ++k) {
            const int id = c->set_geo[gi][k];
            if (id < 0) continue;
            const GeoBuf &gb = c->geos[id];
            c->rho[gi][k] = c->rho_all + off;
            off += (size_t)gb.A;
            if ((rc = dev_alloc(c, &c->phi[gi][k], gb.A * c->esz))) return cleanup(rc);
        }
    // pairs: grid 1 alone, grids 2+3, grids 4+5 (grid 5 alone without grid 4)
    for (int gi = 0; gi < sys->ngal; ++gi) {
        auto add_pair = [&](int a, int b) {
            GeoBuf &gb = c->geos[c->set_geo[gi][a]];
            Pair pr;
            pr.gi = gi; pr.a = a; pr.b = b;
            gb.pairs.push_back(pr);
        };
        if (c->set_geo[gi][0] >= 0) {
            add_pair(0, -1);
            c->geos[c->set_geo[gi][0]].pairs.back().diff = true;
        }
        if (c->set_geo[gi][1] >= 0) add_pair(1, 2);
        if (c->set_geo[gi][3] >= 0) add_pair(3, 4);
        else add_pair(4, -1);
    }
    for (GeoBuf &gb : c->geos)
        for (Pair &pr : gb.pairs) {
            const size_t bytes = (size_t)gb.workN * 2 * c->esz;
            if ((rc = dev_alloc(c, &pr.work, bytes))) return cleanup(rc);
            if (cudaMemsetAsync(pr.work, 0, bytes, c->user) != cudaSuccess)
                return cleanup(fail(PM_E_CUDA, "memset failed"));
            if ((rc = pm_encode_col_maps(pr.work, gb.g.nx, gb.g.ny, gb.g.nz, (int)c->esz, &pr.yfwd, &pr.yinv,
                                         &pr.zmap)))
                return cleanup(rc);
            if (!pr.diff) continue;
            if ((rc = dev_alloc(c, &pr.work2, bytes))) return cleanup(rc);
            if (cudaMemsetAsync(pr.work2, 0, bytes, c->user) != cudaSuccess)
                return cleanup(fail(PM_E_CUDA, "memset failed"));
            if ((rc = pm_encode_col_maps(pr.work2, gb.g.nx, gb.g.ny, gb.g.nz, (int)c->esz, &pr.yfwd2, &pr.yinv2,
                                         &pr.zmap2)))
                return cleanup(rc);
            for (int k = 0; k < 3; ++k)
                if ((rc = dev_alloc(c, &c->fd[pr.gi][k], gb.A * c->esz))) return cleanup(rc);
        }
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(PM_E_CUDA, "cudaEventCreate failed"));
    for (int gi = 0; gi < (int)c->geos.size(); ++gi) {   // shapes: geometries of equal cell counts
        const pm_geometry &g = c->geos[gi].g;
        int si = -1;
        for (int k = 0; k < (int)c->shapes.size(); ++k)
            if (c->shapes[k].nx == g.nx && c->shapes[k].ny == g.ny && c->shapes[k].nz == g.nz) si = k;
        if (si < 0) {
            c->shapes.push_back(ShapeGroup{g.nx, g.ny, g.nz, {}});
            si = (int)c->shapes.size() - 1;
        }
        c->shapes[si].geos.push_back(gi);
    }
    set_units(c, true);
    for (size_t l = 0; l < std::max<size_t>(c->geos.size(), 2); ++l) {
        cudaStream_t b;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess)
            return cleanup(fail(PM_E_CUDA, "cudaStreamCreate failed"));
        c->branch.push_back(b);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return cleanup(fail(PM_E_CUDA, "cudaEventCreate failed"));
        c->ev_join.push_back(e);
    }
    for (GeoBuf &gb : c->geos) {
        if ((rc = dev_alloc(c, &gb.hhat, gb.hatN * c->esz))) return cleanup(rc);
        if ((rc = build_hhat(c, gb))) return cleanup(rc);
    }
    if ((rc = (c->prec == PM_FP32 ? upload_twiddles<float>(c) : upload_twiddles<double>(c)))) return cleanup(rc);

    // system description for the particle kernels
    SysK &hs = c->hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.ngal = sys->ngal;
    hs.rsys2 = (float)(sys->r_sys * sys->r_sys);
    for (int k = 0; k < 3; ++k) hs.sc[k] = sys->sys_centre[k];
    hs.mscale = c->mscale;
    hs.mscale_f = (float)c->mscale;
    for (int k = 0; k < 3; ++k) {
        hs.sc_hi[k] = (float)sys->sys_centre[k];
        hs.sc_lo[k] = (float)(sys->sys_centre[k] - (double)hs.sc_hi[k]);
    }
    for (int gi = 0; gi < sys->ngal; ++gi) {
        const pm_galaxy &G = gals[gi];
        GalK &K = hs.gal[gi];
        K.fine = make_geomk(G.fine);
        K.med = make_geomk(G.medium);
        K.coarse = make_geomk(G.coarse);
        K.rc2 = (float)(G.r_core * G.r_core);
        K.ro2 = (float)(G.r_out * G.r_out);
        K.recentre = G.recentre ? 1 : 0;
        K.sD = G.r_core > 0 ? 24 - ceil_log2(G.r_core) : 0;
        for (int k = 0; k < PM_SETS; ++k) K.rho[k] = (unsigned long long *)c->rho[gi][k];
        K.phi_fine = c->phi[gi][0];
        K.fd_x = c->fd[gi][0];
        K.fd_y = c->fd[gi][1];
        K.fd_z = c->fd[gi][2];
        K.phi_m23 = c->phi[gi][1];
        K.phi_m3 = c->phi[gi][2];
        K.phi_call = geom_present(G.medium) ? c->phi[gi][3] : c->phi[gi][4];
        K.phi_c5 = c->phi[gi][4];
    }
    {   // key layout of the spatial sort
        SortK &so = c->sortk;
        std::memset(&so, 0, sizeof(so));
        long long base = 0;
        for (int gi = 0; gi < sys->ngal; ++gi) {
            const pm_geometry *gg[3] = {&gals[gi].fine, &gals[gi].medium, &gals[gi].coarse};
            for (int r = 0; r < 3; ++r) {
                so.base[gi][r] = base;
                if (!geom_present(*gg[r])) continue;
                int b = 0;
                while ((long long)(gg[r]->nx >> b) * (gg[r]->ny >> b) * (gg[r]->nz >> b) > (1LL << 21)) ++b;
                so.shift[gi][r] = b;
                base += (long long)(gg[r]->nx >> b) * (gg[r]->ny >> b) * (gg[r]->nz >> b);
            }
        }
        so.nkeys = base + 1;
        const long long nb = (so.nkeys + 2047) / 2048;
        if ((rc = dev_alloc(c, (void **)&c->s_count, (size_t)nb * 2048 * 4))) return cleanup(rc);
        if ((rc = dev_alloc(c, (void **)&c->s_bsum, (size_t)nb * 4))) return cleanup(rc);
    }
    if ((rc = dev_alloc(c, (void **)&c->d_sys, sizeof(SysK)))) return cleanup(rc);
    if ((rc = dev_alloc(c, (void **)&c->d_cen, sizeof(CenK)))) return cleanup(rc);
    // centre-of-mass accumulators: 64 rows x 8 galaxies x 4 sums, kept zero
    // between uses by the kernel that consumes them
    if ((rc = dev_alloc(c, (void **)&c->d_csum, sizeof(long long) * 4 * PM_MAX_GALAXIES * 64))) return cleanup(rc);
    if ((rc = dev_alloc(c, (void **)&c->d_err, sizeof(int)))) return cleanup(rc);
    if ((rc = dev_alloc(c, (void **)&c->d_diag, sizeof(double) * 8))) return cleanup(rc);
    if ((rc = dev_alloc(c, (void **)&c->d_cnt, sizeof(unsigned long long)))) return cleanup(rc);
    double cen[3 * PM_MAX_GALAXIES] = {0};
    for (int gi = 0; gi < sys->ngal; ++gi)
        for (int k = 0; k < 3; ++k) cen[3 * gi + k] = gals[gi].centre[k];
    const CenK ck = make_cenk(cen, sys->ngal);
    if (cudaMemcpyAsync(c->d_sys, &hs, sizeof(SysK), cudaMemcpyHostToDevice, c->user) != cudaSuccess ||
        cudaMemcpyAsync(c->d_cen, &ck, sizeof(CenK), cudaMemcpyHostToDevice, c->user) != cudaSuccess ||
        cudaMemsetAsync(c->d_csum, 0, sizeof(long long) * 4 * PM_MAX_GALAXIES * 64, c->user) != cudaSuccess ||
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->user) != cudaSuccess ||
        cudaStreamSynchronize(c->user) != cudaSuccess)
        return cleanup(fail(PM_E_CUDA, "context upload failed: %s", cudaGetErrorString(cudaGetLastError())));
    if ((rc = (c->prec == PM_FP32 ? tune_schedule<float>(c) : tune_schedule<double>(c)))) return cleanup(rc);
    *out = c;
    return PM_OK;
}

void pm_destroy(pm_ctx *c) {
    if (!c) return;
    if (c->user) cudaStreamSynchronize(c->user);
    destroy_graph(c);
    for (cudaStream_t b : c->branch) cudaStreamSynchronize(b);
    for (void *p : c->allocs) cudaFree(p);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaStream_t b : c->branch) cudaStreamDestroy(b);
    for (cudaEvent_t e : c->ev_join) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    delete c;
}

int pm_set_launch_config(pm_ctx *c, int32_t batched, int32_t schedule) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    if ((batched != 0 && batched != 1) || (schedule != 0 && schedule != 1))
        return fail(PM_E_ARG, "batched and schedule must be 0 or 1");
    PM_CK(cudaStreamSynchronize(c->user));
    destroy_graph(c);   // captured with the previous configuration's launches
    set_units(c, batched != 0);
    c->sched = c->units.size() < 2 ? 0 : schedule;
    return PM_OK;
}

int pm_set_stream(pm_ctx *c, void *stream) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    c->user = (cudaStream_t)stream;
    return PM_OK;
}

#define PM_DISPATCH(c, F, ...) ((c)->prec == PM_FP32 ? F<float>(__VA_ARGS__) : F<double>(__VA_ARGS__))

int pm_recentre(pm_ctx *c, const pm_particles *p) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    return PM_DISPATCH(c, enqueue_recentre, c, p, c->user);
}

int pm_recentre_sums(pm_ctx *c, const pm_particles *p) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    return PM_DISPATCH(c, enqueue_recentre, c, p, c->user, 1);
}

int pm_recentre_apply(pm_ctx *c) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    pm_particles none;
    std::memset(&none, 0, sizeof(none));
    return PM_DISPATCH(c, enqueue_recentre, c, &none, c->user, 2);
}

int pm_exchange_buffers(pm_ctx *c, void **rho, int64_t *rho_bytes, void **csum, int64_t *csum_bytes) {
    if (!c || !rho || !rho_bytes || !csum || !csum_bytes) return fail(PM_E_ARG, "ctx or an output is NULL");
    *rho = c->rho_all;
    *rho_bytes = (int64_t)c->rho_bytes;
    *csum = c->d_csum;
    *csum_bytes = (int64_t)(sizeof(long long) * 4 * PM_MAX_GALAXIES * 64);
    return PM_OK;
}

int pm_kick_drift(pm_ctx *c, const pm_particles *p, double dt) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (!std::isfinite(dt)) return fail(PM_E_ARG, "dt not finite");
    return PM_DISPATCH(c, force_impl, c, 0, p, dt, nullptr, nullptr, nullptr, nullptr);
}

int pm_deposit(pm_ctx *c, const pm_particles *p) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    return PM_DISPATCH(c, enqueue_deposit, c, p, c->user);
}

int pm_solve(pm_ctx *c) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    return PM_DISPATCH(c, enqueue_solve, c, c->user, nullptr);
}

int pm_force(pm_ctx *c, const pm_particles *p, void *ax, void *ay, void *az) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (p->n > 0 && (!ax || !ay || !az)) return fail(PM_E_ARG, "acceleration array is NULL");
    return PM_DISPATCH(c, force_impl, c, 1, p, 0.0, ax, ay, az, nullptr);
}

int pm_kick(pm_ctx *c, const pm_particles *p, double dt) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (!std::isfinite(dt)) return fail(PM_E_ARG, "dt not finite");
    return PM_DISPATCH(c, force_impl, c, 2, p, dt, nullptr, nullptr, nullptr, nullptr);
}

int pm_step(pm_ctx *c, const pm_particles *p, double dt, int32_t nsteps) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (nsteps < 0 || !std::isfinite(dt)) return fail(PM_E_ARG, "nsteps < 0 or dt not finite");
    if (nsteps == 0) return PM_OK;
    return PM_DISPATCH(c, step_impl, c, p, dt, nsteps);
}

int pm_sort(pm_ctx *c, const pm_particles *p, int64_t *perm) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (p->n == 0) return PM_OK;
    PM_TRY(ensure_sort_scratch(c, p->n));
    return PM_DISPATCH(c, enqueue_sort, c, p, (long long *)perm, c->user);
}

int pm_set_sort_interval(pm_ctx *c, int32_t k) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    if (k < 0) return fail(PM_E_ARG, "sort interval must be >= 0");
    c->sort_interval = k;
    c->step_count = 0;
    destroy_graph(c);
    return PM_OK;
}

int pm_step_timed(pm_ctx *c, const pm_particles *p, double dt, int32_t nsteps, float *ms_out) {
    if (!c || !ms_out) return fail(PM_E_ARG, "ctx or ms_out is NULL");
    PM_TRY(check_particles(p));
    if (nsteps < 1 || !std::isfinite(dt)) return fail(PM_E_ARG, "nsteps < 1 or dt not finite");
    return PM_DISPATCH(c, step_timed_impl, c, p, dt, nsteps, ms_out);
}

int pm_diagnostics(pm_ctx *c, const pm_particles *p, double dt, double *out) {
    if (!c || !out) return fail(PM_E_ARG, "ctx or out is NULL");
    PM_TRY(check_particles(p));
    PM_TRY(pm_deposit(c, p));
    PM_TRY(pm_solve(c));
    PM_CK(cudaMemsetAsync(c->d_diag, 0, sizeof(double) * 8, c->user));
    PM_TRY(PM_DISPATCH(c, force_impl, c, 3, p, dt, nullptr, nullptr, nullptr, c->d_diag));
    double h[8];
    PM_CK(cudaMemcpyAsync(h, c->d_diag, sizeof(h), cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    for (int k = 0; k < 7; ++k) out[k] = h[k];
    return check_device_error(c);
}

int pm_cic_deposit(pm_ctx *c, const pm_particles *p) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    return PM_DISPATCH(c, cic_deposit_impl, c, p);
}

int pm_cic_force(pm_ctx *c, const pm_particles *p, void *ax, void *ay, void *az) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (p->n > 0 && (!ax || !ay || !az)) return fail(PM_E_ARG, "acceleration array is NULL");
    return PM_DISPATCH(c, cic_field_impl, c, 1, p, 0.0, 0.0, ax, ay, az);
}

int pm_cic_kick_drift(pm_ctx *c, const pm_particles *p, double dt_kick, double dt_drift) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (!std::isfinite(dt_kick) || !std::isfinite(dt_drift)) return fail(PM_E_ARG, "dt not finite");
    return PM_DISPATCH(c, cic_field_impl, c, 0, p, dt_kick, dt_drift, nullptr, nullptr, nullptr);
}

int pm_cic_vjp(pm_ctx *c, const pm_particles *p, const void *ux, const void *uy, const void *uz, void *gx, void *gy,
               void *gz, void *gm) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_particles(p));
    if (p->n > 0 && (!ux || !uy || !uz || !gx || !gy || !gz || !gm))
        return fail(PM_E_ARG, "cotangent or gradient array is NULL");
    if (p->n == 0) return PM_OK;
    return PM_DISPATCH(c, cic_vjp_impl, c, p, ux, uy, uz, gx, gy, gz, gm);
}

int pm_disc_diagnostics(pm_ctx *c, const pm_particles *p, const uint8_t *select, const pm_disc_query *q,
                        double *out) {
    if (!c || !q || !out) return fail(PM_E_ARG, "ctx, query or out is NULL");
    PM_TRY(check_particles(p));
    if (q->gal < 0 || q->gal >= c->sys.ngal) return fail(PM_E_ARG, "no galaxy %d", q->gal);
    if (q->nbins < 1 || q->nbins > DG_MAXBINS) return fail(PM_E_ARG, "nbins must be in 1..%d", DG_MAXBINS);
    if (q->nring < 0 || q->mmax < 0 || (long long)q->nring * q->mmax > DG_MAXRM)
        return fail(PM_E_ARG, "need nring >= 0, mmax >= 0, nring * mmax <= %d", DG_MAXRM);
    if (q->nring > 0 && q->mmax > 0 && !(q->r_ring > 0 && std::isfinite(q->r_ring)))
        return fail(PM_E_ARG, "r_ring must be positive");
    if (!(q->dr >= 0) || !std::isfinite(q->r0) || !std::isfinite(q->dr)) return fail(PM_E_ARG, "bad annulus");
    const pm_disc_query qq = *q;
    pm_disc_query q2 = qq;
    if (q2.mmax == 0) q2.nring = 0;
    return PM_DISPATCH(c, disc_impl, c, p, select, &q2, out);
}

int pm_get_density(pm_ctx *c, int32_t gal, int32_t set, int64_t *host_out) {
    if (!c || !host_out) return fail(PM_E_ARG, "ctx or host_out is NULL");
    if (gal < 0 || gal >= c->sys.ngal || set < 1 || set > PM_SETS || c->set_geo[gal][set - 1] < 0)
        return fail(PM_E_ARG, "no grid %d for galaxy %d", set, gal);
    const GeoBuf &gb = c->geos[c->set_geo[gal][set - 1]];
    PM_CK(cudaMemcpyAsync(host_out, c->rho[gal][set - 1], gb.A * 8, cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    return check_device_error(c);
}

int pm_get_potential(pm_ctx *c, int32_t gal, int32_t set, void *host_out) {
    if (!c || !host_out) return fail(PM_E_ARG, "ctx or host_out is NULL");
    if (gal < 0 || gal >= c->sys.ngal || set < 1 || set > PM_SETS || c->set_geo[gal][set - 1] < 0)
        return fail(PM_E_ARG, "no grid %d for galaxy %d", set, gal);
    const GeoBuf &gb = c->geos[c->set_geo[gal][set - 1]];
    PM_CK(cudaMemcpyAsync(host_out, c->phi[gal][set - 1], gb.A * c->esz, cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    return check_device_error(c);
}

int pm_get_centres(pm_ctx *c, double *host_out) {
    if (!c || !host_out) return fail(PM_E_ARG, "ctx or host_out is NULL");
    PM_CK(cudaMemcpyAsync(host_out, c->d_cen, sizeof(double) * 3 * c->sys.ngal, cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    return PM_OK;
}

int pm_set_centres(pm_ctx *c, const double *host_in) {
    if (!c || !host_in) return fail(PM_E_ARG, "ctx or host_in is NULL");
    const CenK ck = make_cenk(host_in, c->sys.ngal);
    PM_CK(cudaMemcpyAsync(c->d_cen, &ck, sizeof(CenK), cudaMemcpyHostToDevice, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    return PM_OK;
}

int pm_count_lost(pm_ctx *c, const pm_particles *p, int64_t *host_out) {
    if (!c || !host_out) return fail(PM_E_ARG, "ctx or host_out is NULL");
    PM_TRY(check_particles(p));
    PM_CK(cudaMemsetAsync(c->d_cnt, 0, sizeof(unsigned long long), c->user));
    cudaError_t e = (c->prec == PM_FP32) ? pm_launch_count_lost<float>(part_k<float>(p), c->d_cnt, c->user)
                                          : pm_launch_count_lost<double>(part_k<double>(p), c->d_cnt, c->user);
    PM_CK(e);
    unsigned long long h = 0;
    PM_CK(cudaMemcpyAsync(&h, c->d_cnt, sizeof(h), cudaMemcpyDeviceToHost, c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    *host_out = (int64_t)h;
    return check_device_error(c);
}

int pm_selftest_wait_expiry(pm_ctx *c) {
    if (!c) return fail(PM_E_ARG, "ctx is NULL");
    PM_TRY(check_device_error(c));   // starts from a clean flag
    PM_CK(pm_launch_wait_expiry(c->d_err, c->user));
    const int rc = check_device_error(c);
    PM_CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->user));
    PM_CK(cudaStreamSynchronize(c->user));
    return rc;
}

int pm_info(pm_ctx *c, int64_t *out) {
    if (!c || !out) return fail(PM_E_ARG, "ctx or out is NULL");
    int nsets = 0;
    for (const GeoBuf &gb : c->geos) nsets += (int)gb.sets.size();
    out[0] = c->shift;
    out[1] = nsets;
    out[2] = (int64_t)c->geos.size();
    out[3] = (int64_t)c->bytes;
    out[4] = c->units.size() < 2 ? -1 : c->sched;
    out[5] = c->batched ? 1 : 0;
    return PM_OK;
}

}  // extern "C"
