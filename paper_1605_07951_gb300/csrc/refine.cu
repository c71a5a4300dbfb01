// Column kernels of the GMRES-based refinement of rsrr_sample (RSRR_REFINE_GMRES):
// per column c of the n x (N L) FP64 arrays (column c belongs to point
// c / L), restarted GMRES on T(z_j) d = r, right-preconditioned by the
// complex64 band LU (Arnoldi by modified Gram-Schmidt).  Every kernel skips
// the columns of points whose done flag is set.  One CTA per column for the
// reductions; grid-stride loops for the updates.
#include <algorithm>

#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

constexpr int RF_THREADS = 256;

RSRR_DEV double block_sum(double v) {
    __shared__ double red[RF_THREADS / 32];
    for (int off = 16; off; off >>= 1) v += shfl_down(v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < RF_THREADS / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// out[c] = ||W(:, c)||_2
__global__ void rf_norm_kernel(const double2 *__restrict__ W, int64_t n, int L, const int32_t *__restrict__ done,
                               double *__restrict__ out) {
    const int c = blockIdx.x;
    if (done && done[c / L]) return;
    const double2 *w = W + (int64_t)c * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += RF_THREADS) s += w[i].x * w[i].x + w[i].y * w[i].y;
    s = block_sum(s);
    if (threadIdx.x == 0) out[c] = sqrt(s);
}

// h[c] = V(:, c)^H W(:, c)
__global__ void rf_dot_kernel(const double2 *__restrict__ V, const double2 *__restrict__ W, int64_t n, int L,
                              const int32_t *__restrict__ done, double2 *__restrict__ h) {
    const int c = blockIdx.x;
    if (done && done[c / L]) return;
    const double2 *v = V + (int64_t)c * n, *w = W + (int64_t)c * n;
    double re = 0.0, im = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += RF_THREADS) {
        const double2 a = v[i], b = w[i];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    re = block_sum(re);
    im = block_sum(im);
    if (threadIdx.x == 0) h[c] = make_double2(re, im);
}

// W(:, c) = sgn W(:, c) - h[c] V(:, c)   (h NULL: W = sgn W)
__global__ void rf_axpy_kernel(double2 *__restrict__ W, const double2 *__restrict__ V, const double2 *__restrict__ h,
                               double sgn, int64_t n, int ncols, int L, const int32_t *__restrict__ done) {
    const int64_t total = n * ncols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / n);
        if (done && done[c / L]) continue;
        double2 w = W[q];
        w.x *= sgn;
        w.y *= sgn;
        if (h) w = cfms(w, h[c], V[q]);
        W[q] = w;
    }
}

// V(:, c) = W(:, c) / den[c]  (den 0: zero column)
__global__ void rf_scale_kernel(double2 *__restrict__ V, const double2 *__restrict__ W, const double *__restrict__ den,
                                int64_t n, int ncols, int L, const int32_t *__restrict__ done) {
    const int64_t total = n * ncols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / n);
        if (done && done[c / L]) continue;
        const double d = den[c];
        const double2 w = W[q];
        V[q] = d > 0.0 ? make_double2(w.x / d, w.y / d) : make_double2(0.0, 0.0);
    }
}

// X(:, c) += sum_j y[c m + j] Z_j(:, c), Z_j = Z + j * zstride
__global__ void rf_update_kernel(double2 *__restrict__ X, const double2 *__restrict__ Z, int64_t zstride,
                                 const double2 *__restrict__ y, int m, int64_t n, int ncols, int L,
                                 const int32_t *__restrict__ done) {
    const int64_t total = n * ncols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / n);
        if (done && done[c / L]) continue;
        double2 x = X[q];
        for (int j = 0; j < m; ++j) x = cfma(x, y[(size_t)c * m + j], Z[j * zstride + q]);
        X[q] = x;
    }
}

static int rf_grid(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + RF_THREADS - 1) / RF_THREADS, 152 * 16));
}

cudaError_t rf_norm(const double2 *W, int64_t n, int ncols, int L, const int32_t *done, double *out,
                    cudaStream_t s) {
    rf_norm_kernel<<<ncols, RF_THREADS, 0, s>>>(W, n, L, done, out);
    return cudaGetLastError();
}
cudaError_t rf_dot(const double2 *V, const double2 *W, int64_t n, int ncols, int L, const int32_t *done,
                   double2 *h, cudaStream_t s) {
    rf_dot_kernel<<<ncols, RF_THREADS, 0, s>>>(V, W, n, L, done, h);
    return cudaGetLastError();
}
cudaError_t rf_axpy(double2 *W, const double2 *V, const double2 *h, double sgn, int64_t n, int ncols, int L,
                    const int32_t *done, cudaStream_t s) {
    rf_axpy_kernel<<<rf_grid(n * ncols), RF_THREADS, 0, s>>>(W, V, h, sgn, n, ncols, L, done);
    return cudaGetLastError();
}
cudaError_t rf_scale(double2 *V, const double2 *W, const double *den, int64_t n, int ncols, int L,
                     const int32_t *done, cudaStream_t s) {
    rf_scale_kernel<<<rf_grid(n * ncols), RF_THREADS, 0, s>>>(V, W, den, n, ncols, L, done);
    return cudaGetLastError();
}
cudaError_t rf_update(double2 *X, const double2 *Z, int64_t zstride, const double2 *y, int m, int64_t n,
                      int ncols, int L, const int32_t *done, cudaStream_t s) {
    rf_update_kernel<<<rf_grid(n * ncols), RF_THREADS, 0, s>>>(X, Z, zstride, y, m, n, ncols, L, done);
    return cudaGetLastError();
}

}  // namespace rsrr
