// H-hat, the DFT of the even-extended Green's function (Sec. 2.1,
// Eq. eqn:greens and eq:symmetry), built once per geometry in FP64.
//
// H is known on the (nx+1)(ny+1)(nz+1) octant; its doubled-grid extension is
// even along every axis, so its DFT is real, even, and separable into three
// cosine sums over the octant:
//   Hhat(k) = sum_{i=0..n} w_i cos(pi k i / n) H(i),  w_0 = w_n = 1, else 2,
// applied along x, then y, then z.
#include <cuda_runtime.h>
#include "pm_launch.h"

__global__ void k_green_octant(double *h, int nx, int ny, int nz, double q, double h000) {
    const long long P = nx + 1, Q = ny + 1, R = nz + 1, n = P * Q * R;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e % P, j = (e / P) % Q, k = e / (P * Q);
        const double qk = q * (double)k;
        const double r2 = (double)(i * i) + (double)(j * j) + qk * qk;
        h[e] = (e == 0) ? h000 : 1.0 / sqrt(r2);
    }
}

// out[o][m][u] = sum_i cmat[m][i] * in[o][i][u],  m, i in [0, n1)
__global__ void k_axis_transform(const double *__restrict__ in, double *__restrict__ out,
                                 const double *__restrict__ cmat, int n1, long long outer, long long inner) {
    const long long n = outer * n1 * inner;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long u = e % inner, m = (e / inner) % n1, o = e / (inner * n1);
        const double *src = in + o * n1 * inner + u;
        const double *row = cmat + m * n1;
        double s = 0.0;
        for (int i = 0; i < n1; ++i) s = fma(row[i], src[(long long)i * inner], s);
        out[e] = s;
    }
}

static int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 16 ? (b > 0 ? b : 1) : 152LL * 16);
}

cudaError_t pm_green_octant(double *h, int nx, int ny, int nz, double q, double h000, cudaStream_t st) {
    const long long n = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    k_green_octant<<<grid_for(n), 256, 0, st>>>(h, nx, ny, nz, q, h000);
    return cudaGetLastError();
}

cudaError_t pm_axis_transform(const double *in, double *out, const double *cmat, int n1, long long outer,
                              long long inner, cudaStream_t st) {
    k_axis_transform<<<grid_for(outer * n1 * inner), 256, 0, st>>>(in, out, cmat, n1, outer, inner);
    return cudaGetLastError();
}
