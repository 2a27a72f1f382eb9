// pm_potential_static: the isolated-boundary potential of one grid without
// any device allocation.
//
// Some callers cannot call cudaMalloc: code embedded in a host application
// whose device memory is pre-partitioned by its own pool (a cudaMalloc there
// fails, or synchronises the whole device), and plugins that may not allocate
// after start-up.  This entry point serves them: the caller passes the density and the output array, and every
// intermediate (spectrum, H-hat, the FP64 temporaries of the H-hat build and
// the twiddle tables) lives in one file-scope __device__ array of fixed size
// that every GPU loading the library holds until the process exits.
//
// A pass whose bounded wait for a tensor copy expires stops early and sets
// an error word in the scratch.  The call cannot wait for its own work, so
// the last kernel it enqueues checks that word: if set, it fills the output
// with NaN and raises a status word that stays set until
// pm_potential_static_status reads it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pm.h"
#include "pm_launch.h"

#define PM_STATIC_SCRATCH_BYTES (32u << 20)
#define PM_STATIC_MAX_DEVICES 64

// The scratch.  Host code must not hand this name to a kernel: on the host it
// is a stand-in symbol, not a device address; its device address is taken
// with cudaGetSymbolAddress, with the device current, at the start of every
// call (scratch_base).
static __device__ __align__(256) unsigned char g_pm_static_scratch[PM_STATIC_SCRATCH_BYTES];

// The first 256 bytes of the scratch hold the status word (set by an
// expired wait, cleared by pm_potential_static_status); every call's
// intermediates start after it.
#define PM_STATIC_STATUS_BYTES 256u

namespace {

std::mutex g_mu;
void *g_ptr[PM_STATIC_MAX_DEVICES];
bool g_attrs[PM_STATIC_MAX_DEVICES][2];

// Reports through pm_last_error().
int sfail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return pm_internal_fail(code, buf);
}

__global__ void k_static_cosmat(double *c, int n) {
    // c[m][i] = w_i cos(pi m i / n), w_0 = w_n = 1, else 2 (n a power of two)
    const int n1 = n + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 * n1; e += gridDim.x * blockDim.x) {
        const int m = e / n1, i = e % n1;
        const long long r = ((long long)m * i) % (2LL * n);
        c[e] = ((i == 0 || i == n) ? 1.0 : 2.0) * cospi((double)r / (double)n);
    }
}

template <typename T>
__global__ void k_static_twiddles(typename cplx_t<T>::type *tw, int L) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)L, &s, &c);
        tw[m].x = (T)c;
        tw[m].y = (T)(-s);
    }
}

// Last kernel of a call: if a pass's bounded wait expired (*err set), the
// output is filled with NaN and the status word raised (it stays raised
// until pm_potential_static_status clears it).
template <typename T>
__global__ void k_static_settle(const int *err, int *status, T *phi, long long n) {
    if (*(volatile const int *)err == 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(status, 1);
    const T qnan = (T)__int_as_float(0x7fc00000);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        phi[i] = qnan;
}

template <typename T> cudaError_t launch_settle(const int *err, int *status, void *phi, long long n, cudaStream_t st) {
    long long b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    k_static_settle<T><<<(int)b, 256, 0, st>>>(err, status, (T *)phi, n);
    return cudaGetLastError();
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

bool pow2_ok(int n) { return n >= 8 && n <= 256 && (n & (n - 1)) == 0; }

template <typename T>
int run(const int64_t *rho, void *phi, int nx, int ny, int nz, double l_xy, double l_z, double G, double h000,
        int shift, unsigned char *base, cudaStream_t st) {
    typedef typename cplx_t<T>::type C;
    const size_t oct = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    const int nmax = std::max(nx, std::max(ny, nz)) + 1;
    int *status = (int *)base;
    size_t off = PM_STATIC_STATUS_BYTES;
    auto take = [&](size_t bytes) { unsigned char *p = base + off; off += up256(bytes); return p; };
    C *work = (C *)take((size_t)nz * 2 * ny * 2 * nx * sizeof(C));
    T *hhat = (T *)take((size_t)pm_hhat_table_size(nx, ny, nz) * sizeof(T));
    double *h = (double *)take(oct * sizeof(double));
    double *t1 = (double *)take(oct * sizeof(double));
    double *cm = (double *)take((size_t)nmax * nmax * sizeof(double));
    int *err = (int *)take(sizeof(int));
    C *twx = (C *)take((size_t)2 * nx * sizeof(C));
    C *twy = (C *)take((size_t)2 * ny * sizeof(C));
    C *twz = (C *)take((size_t)2 * nz * sizeof(C));

#define SCK(call)                                                                               \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return sfail(PM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

    k_static_twiddles<T><<<1, 256, 0, st>>>(twx, 2 * nx);
    k_static_twiddles<T><<<1, 256, 0, st>>>(twy, 2 * ny);
    k_static_twiddles<T><<<1, 256, 0, st>>>(twz, 2 * nz);
    SCK(cudaGetLastError());
    // H-hat: FP64 octant of H, three cosine sums (x, y, z), scaled into T
    SCK(pm_green_octant(h, nx, ny, nz, l_z / l_xy, h000, st));
    k_static_cosmat<<<64, 256, 0, st>>>(cm, nx);
    SCK(cudaGetLastError());
    SCK(pm_axis_transform(h, t1, cm, nx + 1, (long long)(nz + 1) * (ny + 1), 1, st));
    k_static_cosmat<<<64, 256, 0, st>>>(cm, ny);
    SCK(cudaGetLastError());
    SCK(pm_axis_transform(t1, h, cm, ny + 1, nz + 1, nx + 1, st));
    k_static_cosmat<<<64, 256, 0, st>>>(cm, nz);
    SCK(cudaGetLastError());
    SCK(pm_axis_transform(h, t1, cm, nz + 1, 1, (long long)(ny + 1) * (nx + 1), st));
    SCK(pm_store_hhat<T>(t1, hhat, nx, ny, nz, G / (l_xy * 8.0 * nx * ny * nz), st));

    CUtensorMap yfwd, yinv, zmap;
    if (pm_encode_col_maps(work, nx, ny, nz, (int)sizeof(T), &yfwd, &yinv, &zmap) != PM_OK) return PM_E_CUDA;
    SCK(cudaMemsetAsync(err, 0, sizeof(int), st));
    PairArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rho_a = (const long long *)rho;
    a.rho_b = nullptr;
    a.work = work;
    a.phi_b = nullptr;
    a.phi_sum = phi;
    a.hhat = hhat;
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.scale = std::ldexp(1.0, -shift);
    a.err = err;
    a.tw = twx;
    SCK(pm_launch_xfwd<T>(pm_single_batch(a, nullptr, nullptr), st));
    a.tw = twy;
    SCK(pm_launch_col<T>(pm_single_batch(a, &yfwd, &yinv), COL_YFWD, st));
    a.tw = twz;
    SCK(pm_launch_col<T>(pm_single_batch(a, &zmap, nullptr), COL_ZCONV, st));
    a.tw = twy;
    SCK(pm_launch_col<T>(pm_single_batch(a, &yinv, &yfwd), COL_YINV, st));
    a.tw = twx;
    SCK(pm_launch_xinv<T>(pm_single_batch(a, nullptr, nullptr), st));
    SCK(launch_settle<T>(err, status, phi, (long long)nx * ny * nz, st));
#undef SCK
    return PM_OK;
}

size_t scratch_bytes(int nx, int ny, int nz, size_t esz) {
    const size_t oct = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    const size_t nmax = std::max(nx, std::max(ny, nz)) + 1;
    return PM_STATIC_STATUS_BYTES + up256((size_t)nz * 2 * ny * 2 * nx * 2 * esz) + up256((size_t)pm_hhat_table_size(nx, ny, nz) * esz) +
           2 * up256(oct * 8) +
           up256(nmax * nmax * 8) + up256(sizeof(int)) + up256((size_t)2 * nx * 2 * esz) +
           up256((size_t)2 * ny * 2 * esz) + up256((size_t)2 * nz * 2 * esz);
}

int current_device(int *dev) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return sfail(PM_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (*dev < 0 || *dev >= PM_STATIC_MAX_DEVICES) return sfail(PM_E_ARG, "device %d out of range", *dev);
    return PM_OK;
}

// Set-up, with device `dev` current: the scratch's device address (looked
// up on every call; it is a host-side lookup) and, once per device and
// precision, the kernels' shared-memory limits.  A changed address means a
// new context on the device (after a device reset), whose kernels need their
// attributes set again.
int scratch_base(int dev, int pi, unsigned char **base) {
    std::lock_guard<std::mutex> lk(g_mu);
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pm_static_scratch);
    if (e != cudaSuccess || !p) return sfail(PM_E_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    if (p != g_ptr[dev]) {
        g_ptr[dev] = p;
        g_attrs[dev][0] = g_attrs[dev][1] = false;
    }
    if (pi >= 0 && !g_attrs[dev][pi]) {
        e = pi == 0 ? pm_set_attrs<float>() : pm_set_attrs<double>();
        if (e != cudaSuccess) return sfail(PM_E_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
        g_attrs[dev][pi] = true;
    }
    *base = (unsigned char *)p;
    return PM_OK;
}

}  // namespace

#define PM_STATIC_TRY(expr)         \
    do {                            \
        const int rc_ = (expr);     \
        if (rc_ != PM_OK) return rc_; \
    } while (0)

extern "C" int pm_potential_static(const int64_t *rho, void *phi, int32_t nx, int32_t ny, int32_t nz, double l_xy,
                                   double l_z, double G, double h000, int32_t shift, int32_t precision,
                                   void *stream) {
    if (!rho || !phi) return sfail(PM_E_ARG, "rho or phi is NULL");
    if (precision != PM_FP32 && precision != PM_FP64) return sfail(PM_E_ARG, "precision must be PM_FP32 or PM_FP64");
    if (!pow2_ok(nx) || !pow2_ok(ny) || !pow2_ok(nz))
        return sfail(PM_E_ARG, "nx, ny, nz must be powers of two in [8, 256]");
    if (!(l_xy > 0) || !(l_z > 0) || !std::isfinite(l_xy) || !std::isfinite(l_z) || !std::isfinite(G) ||
        !std::isfinite(h000) || shift < -60 || shift > 1000)
        return sfail(PM_E_ARG, "cell lengths must be positive, G and h000 finite, shift in [-60, 1000]");
    const size_t need = scratch_bytes(nx, ny, nz, precision == PM_FP32 ? 4 : 8);
    if (need > PM_STATIC_SCRATCH_BYTES)
        return sfail(PM_E_ARG, "grid %dx%dx%d needs %zu bytes of scratch; the static scratch holds %u bytes", nx, ny,
                     nz, need, (unsigned)PM_STATIC_SCRATCH_BYTES);
    int dev = 0;
    PM_STATIC_TRY(current_device(&dev));
    unsigned char *base = nullptr;
    PM_STATIC_TRY(scratch_base(dev, precision == PM_FP32 ? 0 : 1, &base));
    cudaStream_t st = (cudaStream_t)stream;
    return precision == PM_FP32 ? run<float>(rho, phi, nx, ny, nz, l_xy, l_z, G, h000, shift, base, st)
                                : run<double>(rho, phi, nx, ny, nz, l_xy, l_z, G, h000, shift, base, st);
}

extern "C" int pm_potential_static_status(void *stream) {
    int dev = 0;
    PM_STATIC_TRY(current_device(&dev));
    unsigned char *base = nullptr;
    PM_STATIC_TRY(scratch_base(dev, -1, &base));
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return sfail(PM_E_CUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    int h = 0;
    e = cudaMemcpy(&h, base, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sfail(PM_E_CUDA, "status read: %s", cudaGetErrorString(e));
    if (!h) return PM_OK;
    e = cudaMemset(base, 0, sizeof(int));
    if (e != cudaSuccess) return sfail(PM_E_CUDA, "status clear: %s", cudaGetErrorString(e));
    return sfail(PM_E_TIMEOUT, "a tensor copy of an allocation-free solve did not complete within its time limit; "
                               "its output was set to NaN");
}

extern "C" int pm_static_selftest_wait_expiry(void *phi, int64_t n, int32_t precision, void *stream) {
    if (!phi || n < 1) return sfail(PM_E_ARG, "phi is NULL or n < 1");
    if (precision != PM_FP32 && precision != PM_FP64) return sfail(PM_E_ARG, "precision must be PM_FP32 or PM_FP64");
    int dev = 0;
    PM_STATIC_TRY(current_device(&dev));
    unsigned char *base = nullptr;
    PM_STATIC_TRY(scratch_base(dev, -1, &base));
    cudaStream_t st = (cudaStream_t)stream;
    int *status = (int *)base;
    int *err = (int *)(base + PM_STATIC_STATUS_BYTES);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = pm_launch_wait_expiry(err, st);
    if (e == cudaSuccess)
        e = precision == PM_FP32 ? launch_settle<float>(err, status, phi, n, st)
                                 : launch_settle<double>(err, status, phi, n, st);
    if (e != cudaSuccess) return sfail(PM_E_CUDA, "self-test launch: %s", cudaGetErrorString(e));
    return PM_OK;
}
