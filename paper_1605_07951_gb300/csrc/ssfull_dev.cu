// Moments of SS-FULL (Section 3.3 with U = I) for the projected NEP on the
// GPU, in FP64:
//
//     A_alpha = sum_q w_q s_q^alpha T_Q(z_q)^{-1},   alpha < 2 K_Q,
//
// with the N_Q trapezoid nodes z_q = gamma + a cos t_q + i b sin t_q,
// t_q = 2 pi (q + 1/2) / N_Q, weights w_q = (-a sin t_q + i b cos t_q) / N_Q
// (Section 5.1) and scaled powers s_q = (z_q - gamma) / rho, rho = max(a, b).
// Nodes are processed in chunks: T_Q(z_q) = sum_i f_i(z_q) P_i is assembled
// for every node of the chunk, factored by the batched complex128 dense LU
// (partial pivoting), T_Q^{-1} obtained by the batched solve with the identity
// as right-hand side, and the weighted inverses summed into the moments in a
// fixed node order.  The Hankel SVD and the small eigenproblem stay on the
// host (ssfull_host.cpp).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "common.cuh"
#include "rsrr_handle.h"

namespace rsrr {

// T[b] = sum_i f[b][i] P_i for the nodes of a chunk (k x k each)
__global__ void tq_assemble_kernel(double2 *__restrict__ T, const double2 *__restrict__ P,
                                   const double2 *__restrict__ f, int m, int64_t kk) {
    const int b = blockIdx.y;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk;
         e += (int64_t)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) acc = cfma(acc, f[(size_t)b * m + i], P[(size_t)i * kk + e]);
        T[(size_t)b * kk + e] = acc;
    }
}

// F[b] = I (k x k) for every node of a chunk
__global__ void tq_identity_kernel(double2 *__restrict__ F, int k) {
    const int b = blockIdx.y;
    const int64_t kk = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk;
         e += (int64_t)gridDim.x * blockDim.x)
        F[(size_t)b * kk + e] = make_double2(e % k == e / k ? 1.0 : 0.0, 0.0);
}

// Acc[alpha] += sum_b c[b][alpha] F[b], nodes summed in order
__global__ void tq_moment_kernel(double2 *__restrict__ Acc, const double2 *__restrict__ F,
                                 const double2 *__restrict__ c, int nb, int nmom, int64_t kk) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kk;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int al = 0; al < nmom; ++al) {
            double2 acc = Acc[(size_t)al * kk + e];
            for (int b = 0; b < nb; ++b) acc = cfma(acc, c[(size_t)b * nmom + al], F[(size_t)b * kk + e]);
            Acc[(size_t)al * kk + e] = acc;
        }
    }
}

static int grid_cap(int64_t work, int threads, int cap) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, cap));
}

// node chunk size: T and F of the chunk within `bytes`, at most NQ
static int ssfull_chunk(int64_t k, int NQ, size_t bytes) {
    const size_t per = sizeof(double2) * (size_t)k * k * 2;
    return (int)std::max<size_t>(1, std::min<size_t>(NQ, bytes / std::max<size_t>(per, 1)));
}

// device bytes of the moment stage for basis size k
size_t ssfull_dev_bytes(int64_t k, int m, int NQ, int KQ) {
    const size_t B = ssfull_chunk(k, NQ, kSsfullChunkBytes);
    const size_t kk = (size_t)k * k;
    const size_t nblk = ((size_t)k + NB_C128 - 1) / NB_C128;
    return sizeof(double2) * (2 * B * kk + (size_t)2 * KQ * kk + B * (m + 2 * KQ) +
                              B * nblk * 2 * NB_C128 * NB_C128) +
           sizeof(int32_t) * (B * k + B) + 8 * 256;
}

rsrr_status Handle::ssfull_moments(const std::vector<std::complex<double>> &fq,
                                   const std::vector<std::complex<double>> &zq,
                                   const std::vector<std::complex<double>> &wq, int KQ,
                                   std::vector<std::vector<std::complex<double>>> &Am) {
    using cplx = std::complex<double>;
    cudaStream_t s = hs;
    const int NQ = (int)zq.size();
    const int nmom = 2 * KQ;
    const int64_t kk = (int64_t)k * k;
    const int B = ssfull_chunk(k, NQ, kSsfullChunkBytes);
    const size_t nblk = ((size_t)k + NB_C128 - 1) / NB_C128;
    const size_t bytes = ssfull_dev_bytes(k, m, NQ, KQ);
    void *buf = nullptr;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&buf, bytes, pool, s) : cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) return fail(RSRR_ENOMEM, "SS-FULL moment buffers", e);
    struct Free {
        Handle *h;
        void *p;
        ~Free() { h->raw_free(p); }
    } guard{this, buf};
    char *p = static_cast<char *>(buf);
    auto take = [&p](size_t b) {
        char *q = p;
        p += (b + 255) / 256 * 256;
        return q;
    };
    double2 *dT = reinterpret_cast<double2 *>(take(sizeof(double2) * B * kk));
    double2 *dF = reinterpret_cast<double2 *>(take(sizeof(double2) * B * kk));
    double2 *dA = reinterpret_cast<double2 *>(take(sizeof(double2) * nmom * kk));
    double2 *df = reinterpret_cast<double2 *>(take(sizeof(double2) * B * m));
    double2 *dc = reinterpret_cast<double2 *>(take(sizeof(double2) * B * nmom));
    double2 *dinv = reinterpret_cast<double2 *>(take(sizeof(double2) * B * nblk * 2 * NB_C128 * NB_C128));
    int32_t *dpiv = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * B * k));
    int32_t *dinfo = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * B));
    if ((size_t)(p - static_cast<char *>(buf)) > bytes) return fail(RSRR_ESTATE, "SS-FULL buffer layout");

    const double rho = std::max(region.a, region.b);
    const cplx gamma(region.center.re, region.center.im);
    std::vector<double2> hf((size_t)B * m), hc((size_t)B * nmom);
    std::vector<int32_t> info(B);
    if ((e = cudaMemsetAsync(dA, 0, sizeof(double2) * nmom * kk, s)) != cudaSuccess)
        return fail(RSRR_ECUDA, "memset", e);
    for (int q0 = 0; q0 < NQ; q0 += B) {
        const int nb = std::min(B, NQ - q0);
        for (int bq = 0; bq < nb; ++bq) {
            const int q = q0 + bq;
            const cplx z = zq[q], w = wq[q];
            for (int i = 0; i < m; ++i) {
                const cplx v = fq[(size_t)q * m + i];
                hf[(size_t)bq * m + i] = make_double2(v.real(), v.imag());
            }
            const cplx sz = (z - gamma) / rho;
            cplx c = w;
            for (int al = 0; al < nmom; ++al) {
                hc[(size_t)bq * nmom + al] = make_double2(c.real(), c.imag());
                c *= sz;
            }
        }
        // (pageable sources: each copy returns once staged, so hf/hc may be refilled)
        if ((e = cudaMemcpyAsync(df, hf.data(), sizeof(double2) * nb * m, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(dc, hc.data(), sizeof(double2) * nb * nmom, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess)
            return fail(RSRR_ECUDA, "SS-FULL coefficients", e);
        tq_assemble_kernel<<<dim3(grid_cap(kk, 256, 1024), nb), 256, 0, s>>>(dT, d_P, df, m, kk);
        tq_identity_kernel<<<dim3(grid_cap(kk, 256, 1024), nb), 256, 0, s>>>(dF, k);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(RSRR_ECUDA, "SS-FULL assemble", e);
        if ((e = launch_dense_lu_c128(dT, dpiv, dinfo, dinv, k, nb, s, &launches)) != cudaSuccess)
            return fail(RSRR_ECUDA, "SS-FULL LU", e);
        if ((e = launch_dense_solve_c128(dT, dpiv, dinv, dF, k, nb, k, nullptr, s)) != cudaSuccess)
            return fail(RSRR_ECUDA, "SS-FULL inverse", e);
        tq_moment_kernel<<<grid_cap(kk, 256, 152 * 8), 256, 0, s>>>(dA, dF, dc, nb, nmom, kk);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(RSRR_ECUDA, "SS-FULL moments", e);
        if ((e = cudaMemcpyAsync(info.data(), dinfo, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(RSRR_ECUDA, "SS-FULL chunk", e);
        launches += 4;
        for (int bq = 0; bq < nb; ++bq)
            if (info[bq] != 0)
                return fail(RSRR_ESINGULAR, "rsrr_solve: projected T_Q singular at a quadrature node");
    }
    Am.assign(nmom, std::vector<cplx>(kk));
    for (int al = 0; al < nmom; ++al)
        if ((e = cudaMemcpyAsync(Am[al].data(), dA + (size_t)al * kk, sizeof(double2) * kk,
                                 cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return fail(RSRR_ECUDA, "SS-FULL moments to host", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(RSRR_ECUDA, "SS-FULL sync", e);
    return RSRR_OK;
}

}  // namespace rsrr
