// RSRR steps 3-4 on the GPU (Section 4.2 last paragraph, Section 4.3 steps
// 3-4): unit-norm columns of S, an orthonormal basis Q of the dominant
// singular subspace of S, and the projected coefficients P_i = Q^H A_i Q.
//
// Truncated SVD through the Gram matrix, all in FP64:
//   G = D^{-1} S^H S D^{-1}            (D = column norms; Hermitian GEMM)
//   G ~ B B^H                           (pivoted Cholesky, stopped when the
//                                        largest remaining diagonal <= floor^2)
//   B^H B = Y Lambda Y^H                (parallel cyclic Jacobi)
//   sigma_j = sqrt(lambda_j),  keep sigma_j > max(delta, floor) sigma_1
//   Q1 = S D^{-1} B Y_k Lambda_k^{-1}  (= S_n V_k Sigma_k^{-1})
//   Q1^H Q1 = Z M Z^H,  Q = Q1 Z M^{-1/2}   (second pass restores
//                                        orthogonality lost in the Gram route)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "rsrr_handle.h"

namespace rsrr {

// ==========================================================================
// FP64 complex GEMM: C = alpha * op(A) * B + beta * C (column major),
// op(A) = A (M x K) or A^H (A is K x M).  64x64 tiles, 256 threads with 4x4
// outputs each, K slabs of 16 through shared memory, optional split-K into a
// workspace (deterministic reduction) and optional upper-tile-only mode for
// Hermitian products (the lower triangle is mirrored afterwards).
// ==========================================================================
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256)
zgemm_kernel(int M, int N, int K, bool conjA, const double2 *__restrict__ A, int64_t lda,
             const double2 *__restrict__ B, int64_t ldb, double2 *__restrict__ Cout, int64_t ldc,
             int kchunk, bool upper_only, double alpha, double beta) {
    const int bm = blockIdx.x, bn = blockIdx.y, ks = blockIdx.z;
    if (upper_only && bm > bn) return;
    __shared__ double2 As[GK][GT + 1];
    __shared__ double2 Bs[GK][GT + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;  // outputs rows tx+16a, cols ty+16b
    const int m0 = bm * GT, n0 = bn * GT;
    const int kbeg = ks * kchunk, kend = min(K, kbeg + kchunk);
    double2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_double2(0.0, 0.0);
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
        // A tile: op(A)(m0+i, k0+kk)
        for (int q = tid; q < GT * GK; q += 256) {
            int i, kk;
            double2 v = make_double2(0.0, 0.0);
            if (conjA) {  // element (kk, i) of A, kk fastest
                kk = q % GK; i = q / GK;
                if (m0 + i < M && k0 + kk < kend) {
                    v = A[(int64_t)(m0 + i) * lda + (k0 + kk)];
                    v.y = -v.y;
                }
            } else {      // element (i, kk) of A, i fastest
                i = q % GT; kk = q / GT;
                if (m0 + i < M && k0 + kk < kend) v = A[(int64_t)(k0 + kk) * lda + (m0 + i)];
            }
            As[kk][i] = v;
        }
        for (int q = tid; q < GT * GK; q += 256) {
            const int kk = q % GK, j = q / GK;
            double2 v = make_double2(0.0, 0.0);
            if (n0 + j < N && k0 + kk < kend) v = B[(int64_t)(n0 + j) * ldb + (k0 + kk)];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            double2 av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = cfma(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
    }
    double2 *Cp = Cout + (int64_t)ks * ldc * N;  // split-K slab (ks = 0 when direct)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = m0 + tx + 16 * a, j = n0 + ty + 16 * b;
            if (i < M && j < N) {
                double2 r = make_double2(alpha * acc[a][b].x, alpha * acc[a][b].y);
                if (beta != 0.0) {
                    const double2 c = Cp[(int64_t)j * ldc + i];
                    r.x = fma(beta, c.x, r.x);
                    r.y = fma(beta, c.y, r.y);
                }
                Cp[(int64_t)j * ldc + i] = r;
            }
        }
}

// C = alpha * sum_s W[s] + beta * C over the split-K slabs (fixed order)
__global__ void splitk_reduce_kernel(double2 *__restrict__ C, int64_t ldc,
                                     const double2 *__restrict__ W, int M, int N, int S,
                                     double2 alpha, double2 beta, bool upper_only) {
    const int64_t total = (int64_t)M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % M), j = (int)(q / M);
        if (upper_only && (i / GT) > (j / GT)) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int t = 0; t < S; ++t) s = cadd(s, W[(int64_t)t * M * N + (int64_t)j * M + i]);
        double2 c = C[(int64_t)j * ldc + i];
        double2 r = cmul(alpha, s);
        if (beta.x != 0.0 || beta.y != 0.0) r = cfma(r, beta, c);
        C[(int64_t)j * ldc + i] = r;
    }
}

// lower triangle <- conj(upper) for Hermitian results computed by tiles
__global__ void hermitian_mirror_kernel(double2 *__restrict__ C, int64_t ldc, int n) {
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        if (i > j) {
            double2 v = C[(int64_t)i * ldc + j];
            C[(int64_t)j * ldc + i] = make_double2(v.x, -v.y);
        }
    }
}

static int grid1d(int64_t work, int threads = 256) {
    int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

// workspace-backed GEMM: chooses split-K so that enough CTAs run
struct Gemm {
    double2 *ws = nullptr;
    size_t ws_elems = 0;
    int64_t *counter = nullptr;
    Handle *timer = nullptr;  // records events around every call when set
    int method = RSRR_GEMM_FP64;
    void *ows = nullptr;      // work space of the sliced tensor-core products
    size_t ows_bytes = 0;
    unsigned int *tmo = nullptr;  // the handle's status word of bounded waits that ran out
    cudaError_t run(int M, int N, int K, bool conjA, const double2 *A, int64_t lda,
                    const double2 *B, int64_t ldb, double2 *C, int64_t ldc, cudaStream_t s,
                    bool hermitian = false, double alpha = 1.0, double beta = 0.0) {
        if (M <= 0 || N <= 0) return cudaSuccess;
        const double flops = hermitian ? 8.0 * (double)M * (M + 1) / 2 * K : 8.0 * M * N * (double)K;
        const bool legacy = method == RSRR_GEMM_OZAKI_MMA;
        const bool sliced = ows && K > 0 &&
                            (method == RSRR_GEMM_OZAKI || legacy ||
                             (method == RSRR_GEMM_AUTO && flops >= 1073741824.0));
        if (sliced) {
            cudaError_t e;
            cudaEvent_t ev1 = nullptr;
            if (timer) {
                cudaEvent_t ev0;
                if ((e = timer->gemm_event(&ev0)) != cudaSuccess) return e;
                if ((e = timer->gemm_event(&ev1)) != cudaSuccess) return e;
                if ((e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
                timer->gemm_flops += flops;
            }
            e = ozaki_zgemm(M, N, K, conjA, A, lda, B, ldb, C, ldc, alpha, beta, hermitian, ows,
                            ows_bytes, s, counter, timer ? &timer->tc_pool : nullptr,
                            timer ? &timer->tc_flops : nullptr, legacy, tmo);
            if (e == cudaSuccess && timer) e = cudaEventRecord(ev1, s);
            return e;
        }
        const int tm = (M + GT - 1) / GT, tn = (N + GT - 1) / GT;
        int64_t tiles = hermitian ? (int64_t)tm * (tm + 1) / 2 : (int64_t)tm * tn;
        int splits = 1;
        const int64_t target = 152 * 2;
        if (tiles < target && K > 4 * GK) {
            splits = (int)std::min<int64_t>((target + tiles - 1) / tiles, (K + 255) / 256);
            while (splits > 1 && (size_t)splits * M * N > ws_elems) --splits;
        }
        if (K <= 0) splits = 1;
        if (splits > 1 && (size_t)splits * M * N > ws_elems) splits = 1;
        int kchunk = (K + splits - 1) / splits;
        kchunk = ((kchunk + GK - 1) / GK) * GK;
        if (kchunk < GK) kchunk = GK;
        splits = std::max(1, (K + kchunk - 1) / kchunk);
        dim3 grid(tm, tn, splits);
        cudaError_t e;
        cudaEvent_t ev1 = nullptr;
        if (timer) {
            cudaEvent_t ev0;
            if ((e = timer->gemm_event(&ev0)) != cudaSuccess) return e;
            if ((e = timer->gemm_event(&ev1)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
            timer->gemm_flops += flops;
        }
        if (counter) *counter += 1 + (splits == 1 ? 0 : 1) + (hermitian ? 1 : 0);
        if (splits == 1) {  // direct: the kernel writes C itself
            zgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, conjA, A, lda, B, ldb, C, ldc, kchunk,
                                              hermitian, alpha, beta);
        } else {
            zgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, conjA, A, lda, B, ldb, ws, M, kchunk,
                                              hermitian, 1.0, 0.0);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            splitk_reduce_kernel<<<grid1d((int64_t)M * N), 256, 0, s>>>(
                C, ldc, ws, M, N, splits, make_double2(alpha, 0.0), make_double2(beta, 0.0),
                hermitian);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (hermitian) {
            hermitian_mirror_kernel<<<grid1d((int64_t)M * M), 256, 0, s>>>(C, ldc, M);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && timer) e = cudaEventRecord(ev1, s);
        return e;
    }
};

cudaError_t fp64_gemm(int M, int N, int K, bool conjA, const double2 *A, int64_t lda, const double2 *B,
                      int64_t ldb, double2 *C, int64_t ldc, double alpha, double beta, cudaStream_t s) {
    Gemm g;  // no work space: always the direct path
    return g.run(M, N, K, conjA, A, lda, B, ldb, C, ldc, s, false, alpha, beta);
}

// ==========================================================================
// column norms and scalings
// ==========================================================================
__global__ void colnorm_kernel(double *__restrict__ nrm, const double2 *__restrict__ X, int64_t n) {
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 v = X[(int64_t)c * n + i];
        s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    for (int off = 16; off; off >>= 1) s += shfl_down(s, off);
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += w[q];
        nrm[c] = sqrt(r);
    }
}

// G(i,j) /= (d_i d_j)
__global__ void gram_scale_kernel(double2 *__restrict__ G, const double *__restrict__ d, int n) {
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        const double s = 1.0 / (d[i] * d[j]);
        G[q].x *= s;
        G[q].y *= s;
    }
}

// W(i, j) *= rs[i] * cs[j]   (rs or cs may be null)
__global__ void scale_rc_kernel(double2 *__restrict__ W, int64_t ld, int M, int N,
                                const double *__restrict__ rs, const double *__restrict__ cs,
                                bool rs_inverse, bool cs_inv_sqrt) {
    const int64_t total = (int64_t)M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % M), j = (int)(q / M);
        double s = 1.0;
        if (rs) s *= rs_inverse ? 1.0 / rs[i] : rs[i];
        if (cs) s *= cs_inv_sqrt ? 1.0 / sqrt(cs[j]) : 1.0 / cs[j];
        double2 &w = W[(int64_t)j * ld + i];
        w.x *= s;
        w.y *= s;
    }
}

__global__ void diag_real_kernel(double *__restrict__ d, const double2 *__restrict__ G, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = G[(int64_t)i * n + i].x;
}

// ==========================================================================
// Bounded grid-wide barrier for cooperative launches (all CTAs co-resident).
// bar[0] arrivals, bar[1] generation, bar[2] error flag.  A CTA that waits
// more than 2^24 polls (~2 s) sets the error flag; every CTA then stops.
// Returns false once the flag is set.
// ==========================================================================
constexpr long long GRID_WAIT_LIMIT = 1LL << 24;

RSRR_DEV bool grid_sync(unsigned int *bar, unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vb = bar;
        const unsigned int gen = vb[1];
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (vb[1] == gen) {
                if (vb[2]) { ok = 0; break; }
                if (++it > GRID_WAIT_LIMIT) { atomicExch(bar + 2, 1u); ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && !vb[2];
    }
    __syncthreads();
    return s_ok != 0;
}

// block-wide argmax of d (first index on ties); every CTA computes it
RSRR_DEV void block_argmax(const double *__restrict__ d, int n, double &bv, int &bi) {
    __shared__ double s_v[256];
    __shared__ int s_i[256];
    double v = -1.0;
    int ix = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = d[i];
        if (x > v || (x == v && i < ix)) { v = x; ix = i; }
    }
    s_v[threadIdx.x] = v;
    s_i[threadIdx.x] = ix;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double ov = s_v[threadIdx.x + w];
            const int oi = s_i[threadIdx.x + w];
            if (ov > s_v[threadIdx.x] || (ov == s_v[threadIdx.x] && oi < s_i[threadIdx.x])) {
                s_v[threadIdx.x] = ov;
                s_i[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    bv = s_v[0];
    bi = s_i[0];
    __syncthreads();
}

// Pivoted Cholesky G ~ L L^H in one cooperative launch (left-looking; one
// grid barrier per column).  state[0] = stopped, state[1] = kc; pivots
// (optional): the row of G chosen in each column.
__global__ void __launch_bounds__(256)
pchol_persistent_kernel(const double2 *__restrict__ G, int n, double2 *__restrict__ Lm,
                        double *__restrict__ dbuf, double tau, int32_t *__restrict__ state,
                        unsigned int *__restrict__ bar, int32_t *__restrict__ pivots) {
    for (int j = 0; j < n; ++j) {
        const double *dprev = dbuf + (j & 1) * n;
        double *dnext = dbuf + ((j + 1) & 1) * n;
        double dp;
        int p;
        block_argmax(dprev, n, dp, p);
        if (!(dp > tau)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) { state[1] = j; state[0] = 1; }
            return;
        }
        if (pivots && blockIdx.x == 0 && threadIdx.x == 0) pivots[j] = p;
        const double sq = sqrt(dp);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            double2 l = make_double2(0.0, 0.0);
            double dn = dprev[i];
            if (i == p) {
                l = make_double2(sq, 0.0);
                dn = -1.0;
            } else if (dn >= 0.0) {
                double2 s = G[(int64_t)p * n + i];
                for (int t = 0; t < j; ++t) {
                    const double2 a = Lm[(int64_t)t * n + i], b = Lm[(int64_t)t * n + p];
                    s.x -= a.x * b.x + a.y * b.y;
                    s.y -= a.y * b.x - a.x * b.y;
                }
                l = make_double2(s.x / sq, s.y / sq);
                dn = fmax(0.0, dn - (l.x * l.x + l.y * l.y));
            }
            Lm[(int64_t)j * n + i] = l;
            dnext[i] = dn;
        }
        if (!grid_sync(bar, gridDim.x)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) { state[1] = n; state[0] = 1; }
}

// ==========================================================================
// Parallel cyclic Jacobi for a Hermitian k x k matrix: one launch per round
// of the round-robin ordering (k' = k rounded up to even, k'-1 rounds a
// sweep).  Each thread owns a 2x2 block (pair a, pair b) of H and rewrites it
// as J_a^H H J_b, reading the old matrix and writing the new one (double
// buffer); the rotations come from the old matrix.  Y <- Y J in place.
// Rotation for [[alpha, beta], [conj(beta), gamma]], beta = |beta| e^{i phi}:
//   tau = (gamma - alpha) / (2|beta|), t = sign(tau)/(|tau| + sqrt(1+tau^2)),
//   c = 1/sqrt(1+t^2), s = t c,  J = [[c, s e^{i phi}], [-s e^{-i phi}, c]].
// ==========================================================================
struct Rot {
    double c;
    double2 se;  // s e^{i phi}
};

RSRR_DEV void pair_of(int r, int a, int kp, int &p, int &q) {
    if (a == 0) {
        p = kp - 1;
        q = r;
    } else {
        p = (r + a) % (kp - 1);
        q = (r - a + (kp - 1)) % (kp - 1);
    }
    if (p > q) { const int t = p; p = q; q = t; }
}

RSRR_DEV Rot rot_of(const double2 *__restrict__ H, int k, int p, int q) {
    Rot R;
    R.c = 1.0;
    R.se = make_double2(0.0, 0.0);
    if (p >= k || q >= k) return R;
    const double al = H[(int64_t)p * k + p].x, ga = H[(int64_t)q * k + q].x;
    const double2 be = H[(int64_t)q * k + p];  // H(p, q)
    const double ab = hypot(be.x, be.y);
    if (ab <= 1e-300 || ab <= 1e-18 * sqrt(fabs(al * ga))) return R;
    const double tau = (ga - al) / (2.0 * ab);
    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
    R.c = c;
    R.se = make_double2(s * be.x / ab, s * be.y / ab);
    return R;
}

// One round of the round-robin ordering, grid-stride over the 2x2 blocks and
// the rows of Y.  Every CTA first computes the round's np rotations (one per
// pair, from the old matrix) into shared memory `srot`, so that the FP64
// square roots and divisions run once per pair rather than once per block.
RSRR_DEV void jacobi_round(const double2 *__restrict__ Hold, double2 *__restrict__ Hnew,
                           double2 *__restrict__ Y, int k, int kp, int r, Rot *__restrict__ srot) {
    const int np = kp / 2;
    const int64_t nblk = (int64_t)np * np;
    const int64_t nY = (int64_t)k * np;
    for (int a = threadIdx.x; a < np; a += blockDim.x) {
        int p, q;
        pair_of(r, a, kp, p, q);
        srot[a] = rot_of(Hold, k, p, q);
    }
    __syncthreads();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nblk + nY;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q < nblk) {
            const int a = (int)(q % np), b = (int)(q / np);
            int pa, qa, pb, qb;
            pair_of(r, a, kp, pa, qa);
            pair_of(r, b, kp, pb, qb);
            const Rot Ra = srot[a], Rb = srot[b];
            const bool va = qa < k, vb = qb < k;
            double2 h00 = (pa < k && pb < k) ? Hold[(int64_t)pb * k + pa] : make_double2(0, 0);
            double2 h01 = (pa < k && vb) ? Hold[(int64_t)qb * k + pa] : make_double2(0, 0);
            double2 h10 = (va && pb < k) ? Hold[(int64_t)pb * k + qa] : make_double2(0, 0);
            double2 h11 = (va && vb) ? Hold[(int64_t)qb * k + qa] : make_double2(0, 0);
            const double cb = Rb.c;
            const double2 sb = Rb.se, sbc = make_double2(-sb.x, sb.y);
            double2 t00 = cadd(make_double2(h00.x * cb, h00.y * cb), cmul(h01, sbc));
            double2 t01 = cadd(cmul(h00, sb), make_double2(h01.x * cb, h01.y * cb));
            double2 t10 = cadd(make_double2(h10.x * cb, h10.y * cb), cmul(h11, sbc));
            double2 t11 = cadd(cmul(h10, sb), make_double2(h11.x * cb, h11.y * cb));
            const double ca = Ra.c;
            const double2 sa = Ra.se, msa = make_double2(-sa.x, -sa.y), sac = make_double2(sa.x, -sa.y);
            double2 n00 = cadd(make_double2(t00.x * ca, t00.y * ca), cmul(msa, t10));
            double2 n01 = cadd(make_double2(t01.x * ca, t01.y * ca), cmul(msa, t11));
            double2 n10 = cadd(cmul(sac, t00), make_double2(t10.x * ca, t10.y * ca));
            double2 n11 = cadd(cmul(sac, t01), make_double2(t11.x * ca, t11.y * ca));
            if (a == b) {
                n00.y = 0.0;
                n11.y = 0.0;
                if (Ra.se.x != 0.0 || Ra.se.y != 0.0) {
                    n01 = make_double2(0.0, 0.0);
                    n10 = make_double2(0.0, 0.0);
                }
            }
            if (pa < k && pb < k) Hnew[(int64_t)pb * k + pa] = n00;
            if (pa < k && vb) Hnew[(int64_t)qb * k + pa] = n01;
            if (va && pb < k) Hnew[(int64_t)pb * k + qa] = n10;
            if (va && vb) Hnew[(int64_t)qb * k + qa] = n11;
        } else {
            const int64_t w = q - nblk;
            const int i = (int)(w % k), b = (int)(w / k);
            int pb, qb;
            pair_of(r, b, kp, pb, qb);
            if (qb >= k) continue;
            const Rot Rb = srot[b];
            const double2 yp = Y[(int64_t)pb * k + i], yq = Y[(int64_t)qb * k + i];
            const double2 sbc = make_double2(-Rb.se.x, Rb.se.y);
            Y[(int64_t)pb * k + i] = cadd(make_double2(yp.x * Rb.c, yp.y * Rb.c), cmul(yq, sbc));
            Y[(int64_t)qb * k + i] = cadd(cmul(yp, Rb.se), make_double2(yq.x * Rb.c, yq.y * Rb.c));
        }
    }
}

// Whole cyclic Jacobi in one cooperative launch: Y = I, then sweeps of
// kp-1 rounds (grid barrier after each), convergence test after each sweep
// (off(H)^2 <= tol2 * diag(H)^2 from per-CTA partial sums in acc, one slot
// pair per CTA, added in CTA order).  The final matrix is copied back into
// H0.  state[0] = sweeps run.
__global__ void __launch_bounds__(256)
jacobi_persistent_kernel(double2 *__restrict__ H0, double2 *__restrict__ H1,
                         double2 *__restrict__ Y, int k, int max_sweeps, double tol2,
                         double *__restrict__ acc, int32_t *__restrict__ state,
                         unsigned int *__restrict__ bar) {
    const int kp = k + (k & 1);
    const int64_t kk = (int64_t)k * k;
    extern __shared__ Rot srot[];  // kp / 2 rotations of the current round
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < kk;
         q += (int64_t)gridDim.x * blockDim.x)
        Y[q] = make_double2((q % k) == (q / k) ? 1.0 : 0.0, 0.0);
    if (!grid_sync(bar, gridDim.x)) return;
    double2 *a = H0, *b = H1;
    int sweeps = 0;
    if (k > 1) {
        for (int sw = 0; sw < max_sweeps; ++sw) {
            for (int r = 0; r < kp - 1; ++r) {
                jacobi_round(a, b, Y, k, kp, r, srot);
                if (!grid_sync(bar, gridDim.x)) return;
                double2 *t = a; a = b; b = t;
            }
            ++sweeps;
            double off = 0.0, dia = 0.0;
            for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < kk;
                 q += (int64_t)gridDim.x * blockDim.x) {
                const double2 v = a[q];
                const double m2 = v.x * v.x + v.y * v.y;
                if ((q % k) == (q / k)) dia += m2; else off += m2;
            }
            // deterministic reduction: per-CTA partials in fixed slots, summed
            // in CTA order by every CTA after the barrier
            __shared__ double s_off[8], s_dia[8];
            for (int o = 16; o; o >>= 1) {
                off += shfl_down(off, o);
                dia += shfl_down(dia, o);
            }
            if ((threadIdx.x & 31) == 0) { s_off[threadIdx.x >> 5] = off; s_dia[threadIdx.x >> 5] = dia; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double a = 0.0, b2 = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += s_off[w]; b2 += s_dia[w]; }
                acc[2 * blockIdx.x] = a;
                acc[2 * blockIdx.x + 1] = b2;
            }
            if (!grid_sync(bar, gridDim.x)) return;
            double o2 = 0.0, d2 = 0.0;
            for (int c = 0; c < (int)gridDim.x; ++c) {
                o2 += *((volatile double *)(acc + 2 * c));
                d2 += *((volatile double *)(acc + 2 * c + 1));
            }
            const bool done = o2 <= tol2 * d2;
            if (!grid_sync(bar, gridDim.x)) return;  // acc is rewritten next sweep
            if (done) break;
        }
    }
    if (a != H0) {
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < kk;
             q += (int64_t)gridDim.x * blockDim.x)
            H0[q] = a[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) state[0] = sweeps;
}

// eigenvalues = real diagonal; order[r] = index of the r-th largest (ties by index);
// vals[r] sorted descending.  One CTA.
__global__ void sort_desc_kernel(const double2 *__restrict__ H, int k, int32_t *__restrict__ order,
                                 double *__restrict__ vals) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double vi = H[(int64_t)i * k + i].x;
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const double vj = H[(int64_t)j * k + j].x;
            if (vj > vi || (vj == vi && j < i)) ++rank;
        }
        order[rank] = i;
        vals[rank] = vi;
    }
}

// Dst(:, r) = Src(:, order[r]) for r < cols
__global__ void gather_cols_kernel(double2 *__restrict__ Dst, const double2 *__restrict__ Src,
                                   int64_t rows, int cols, const int32_t *__restrict__ order) {
    const int64_t total = rows * cols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q % rows;
        const int r = (int)(q / rows);
        Dst[q] = Src[(int64_t)order[r] * rows + i];
    }
}

// ==========================================================================
// Y = A_q X for the real CSR matrix A_q (term q of the shared pattern), X n x k
// ==========================================================================
__global__ void spmm_kernel(double2 *__restrict__ Y, const double2 *__restrict__ X,
                            const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx,
                            const double *__restrict__ vals, int n, int k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    double2 s = make_double2(0.0, 0.0);
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const double a = vals[e];
        const double2 x = X[(int64_t)c * n + col_idx[e]];
        s.x = fma(a, x.x, s.x);
        s.y = fma(a, x.y, s.y);
    }
    Y[(int64_t)c * n + i] = s;
}

// ==========================================================================
// orchestration
// ==========================================================================
struct ProjWs {
    double *norms;      // NL
    double2 *G;         // NL x NL
    double2 *Lm;        // NL x NL (pivoted Cholesky factor, first kc columns)
    double *dbuf;       // 2 x NL
    int32_t *state;     // 2 + NL
    double2 *H, *H2;    // NL x NL each (Jacobi double buffer)
    double2 *Y;         // NL x NL eigenvectors
    double2 *Ysort;     // NL x NL
    int32_t *order;     // NL
    double *evals;      // NL
    int32_t *conv;      // 1
    double *acc;        // 2
    double2 *W;         // NL x NL
    double2 *Q1;        // n x NL
    double2 *Ytmp;      // n x NL (A_q Q)
    double2 *gws;       // GEMM workspace
    size_t gws_elems;
    double2 *C;         // NL x NL coefficients of the deflation
    unsigned int *bar;  // grid barrier of the cooperative kernels
    double *jacc;       // per-sweep convergence sums of the Jacobi kernel
    void *ows;          // sliced tensor-core GEMM work space
    size_t ows_bytes;
    double2 *Qall;      // n x NL basis
    double2 *P;         // RSRR_MAX_TERMS x NL x NL projected coefficients
    char *end;
};

template <typename T> static T *carve(char *&p, size_t count) {
    T *r = reinterpret_cast<T *>(p);
    p += ((sizeof(T) * count + 255) / 256) * 256;
    return r;
}

#define PK(expr, what)                                                   \
    do {                                                                 \
        cudaError_t _e = (expr);                                         \
        if (_e != cudaSuccess) return fail(RSRR_ECUDA, what, _e);        \
    } while (0)

// Cooperative launch helper: as many CTAs as can be co-resident (<= cap),
// `smem` bytes of dynamic shared memory each.
template <typename K, typename... Args>
static cudaError_t launch_coop_smem(K kern, int cap, size_t smem, cudaStream_t s, Args... args) {
    int dev = 0, nsm = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && smem > 48 * 1024) {
        const int limit = smem_optin_limit();
        if (smem > (size_t)limit) return cudaErrorInvalidConfiguration;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    }
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem);
    if (e != cudaSuccess) return e;
    int grid = std::max(1, std::min(cap, nsm * std::max(per, 1)));
    void *argv[] = {(void *)&args...};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(256), argv, smem, s);
}
template <typename K, typename... Args>
static cudaError_t launch_coop(K kern, int cap, cudaStream_t s, Args... args) {
    return launch_coop_smem(kern, cap, 0, s, args...);
}

// Jacobi on the k x k Hermitian matrix in ws.H (overwritten with its
// eigenvalues on the diagonal); eigenvalues sorted descending into
// ws.evals, eigenvectors (same order) into ws.Ysort.  One cooperative
// launch plus the sort; a barrier timeout is reported through ws.bar[2].
static cudaError_t jacobi_eig(ProjWs &ws, int k, cudaStream_t s, int64_t *counter,
                              int max_sweeps = 30) {
    cudaError_t e = cudaMemsetAsync(ws.bar, 0, sizeof(unsigned int) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.jacc, 0, sizeof(double) * 2 * 4096, s);
    if (e != cudaSuccess) return e;
    const double tol2 = 1e-30;  // off(H) <= 1e-15 ||diag(H)||
    const int64_t work = (int64_t)(k + 1) / 2 * ((k + 1) / 2) + (int64_t)k * ((k + 1) / 2);
    const size_t smem = sizeof(Rot) * (size_t)((k + 1) / 2);
    // at most one CTA per SM: the round's work is FP64-bound per SM either way,
    // and fewer arrivals make the grid barrier after every round cheaper
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = launch_coop_smem(jacobi_persistent_kernel, (int)std::min<int64_t>((work + 255) / 256, nsm), smem,
                         s, ws.H, ws.H2, ws.Y, k, max_sweeps, tol2, ws.jacc, ws.state + 1, ws.bar);
    if (e != cudaSuccess) return e;
    sort_desc_kernel<<<1, 256, 0, s>>>(ws.H, k, ws.order, ws.evals);
    gather_cols_kernel<<<grid1d((int64_t)k * k), 256, 0, s>>>(ws.Ysort, ws.Y, k, k, ws.order);
    *counter += 3;
    return cudaGetLastError();
}

// Scale the columns of X into Sn: Sn(:, c) = X(:, c) / d[c]
__global__ void scale_cols_kernel(double2 *__restrict__ Sn, const double2 *__restrict__ X,
                                  const double *__restrict__ d, int64_t n, int ncol) {
    const int64_t total = n * ncol;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const double s = 1.0 / d[q / n];
        Sn[q] = make_double2(X[q].x * s, X[q].y * s);
    }
}

__global__ void max_diag_kernel(double *__restrict__ out, const double2 *__restrict__ G, int n) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, G[(int64_t)i * n + i].x);
    for (int off = 16; off; off >>= 1) m = fmax(m, shfl_down(m, off));
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, w[q]);
        out[0] = r;
    }
}

// d[c] = G(c,c) - sum_j |C(j,c)|^2 (clamped at 0): squared column norms of
// R - Q C for C = Q^H R with orthonormal Q, without forming it
__global__ void remainder_norm_kernel(double *__restrict__ d, const double2 *__restrict__ G,
                                      const double2 *__restrict__ Cm, int kb, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s = G[(int64_t)c * n + c].x;
    for (int j = 0; j < kb; ++j) {
        const double2 v = Cm[(int64_t)c * kb + j];
        s -= v.x * v.x + v.y * v.y;
    }
    d[c] = fmax(s, 0.0);
}

__global__ void max_vec_kernel(double *__restrict__ out, const double *__restrict__ v, int n) {
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
    for (int off = 16; off; off >>= 1) m = fmax(m, shfl_down(m, off));
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, w[q]);
        out[0] = r;
    }
}

// Orthonormalisation of a block Qb (k columns) from its Gram G2 = Qb^H Qb by
// Cholesky QR with column pivoting: G2 = P L L^H P^T (pivoted Cholesky,
// stopped when the largest remaining diagonal falls below the threshold);
// with T = the leading kc x kc block of L in pivot order (lower triangular,
// real positive diagonal), Qb's pivot columns times T^{-H} have the Gram
// T^{-1} (T T^H) T^{-H} = I.  X (k x kc) = S T^{-H}, S the pivot selection.

// T(i, j) = L(piv[i], j) for j <= i, else 0 (kc x kc, column major)
__global__ void tri_from_pchol_kernel(double2 *__restrict__ T, const double2 *__restrict__ L,
                                      const int32_t *__restrict__ piv, int k, int kc) {
    const int64_t total = (int64_t)kc * kc;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % kc), j = (int)(q / kc);
        T[q] = j <= i ? L[(int64_t)j * k + piv[i]] : make_double2(0.0, 0.0);
    }
}

// W = T^{-1} for lower triangular T with a real positive diagonal: one warp
// per column j, forward substitution w_i = ([i == j] - sum_{j<=t<i} T(i,t) w_t)
// / T(i,i), the sum split over the lanes (fixed order: lane partials, then a
// shuffle tree)
__global__ void tri_inverse_lower_kernel(double2 *__restrict__ W, const double2 *__restrict__ T, int kc) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= kc) return;
    double2 *w = W + (int64_t)j * kc;
    for (int i = lane; i < j; i += 32) w[i] = make_double2(0.0, 0.0);
    for (int i = j; i < kc; ++i) {
        double2 acc = make_double2(0.0, 0.0);
        for (int t = j + lane; t < i; t += 32) acc = cfma(acc, T[(int64_t)t * kc + i], w[t]);
        for (int off = 16; off; off >>= 1) {
            acc.x += shfl_down(acc.x, off);
            acc.y += shfl_down(acc.y, off);
        }
        if (lane == 0) {
            const double d = T[(int64_t)i * kc + i].x;
            const double rx = (i == j ? 1.0 : 0.0) - acc.x, ry = -acc.y;
            w[i] = make_double2(rx / d, ry / d);
        }
        __syncwarp();
    }
}

// X (k x kc, column major, zeroed before) = S W^H: X(piv[i], j) = conj(W(j, i))
__global__ void scatter_inverse_fill_kernel(double2 *__restrict__ X, const double2 *__restrict__ W,
                                            const int32_t *__restrict__ piv, int k, int kc) {
    const int64_t total = (int64_t)kc * kc;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % kc), j = (int)(q / kc);  // X(piv[i], j) = conj(W(j, i))
        const double2 v = W[(int64_t)i * kc + j];
        X[(int64_t)j * k + piv[i]] = make_double2(v.x, -v.y);
    }
}

// Work space of the sliced products: the Gram matrix of the n x NL block in
// one piece (the other products of the sparse kind need less), capped at
// 8 GiB; a product that needs more runs in chunks of K.
static size_t ozaki_ws_bytes(int NL, int64_t n) {
    const int nc = (int)std::min<int64_t>(n, INT32_MAX / 2);
    return std::min(ozaki_workspace_bytes(NL, NL, nc, true), (size_t)8 << 30);
}

// Workspace layout of the projection stage (carved from one allocation).
static void carve_ws(char *cp, ProjWs &ws, int NL, int64_t n, int terms) {
    const size_t NL2 = (size_t)NL * NL;
    ws.norms = carve<double>(cp, NL);
    ws.G = carve<double2>(cp, NL2);
    ws.Lm = carve<double2>(cp, NL2);
    ws.dbuf = carve<double>(cp, 2 * NL);
    ws.state = carve<int32_t>(cp, 2 + NL);
    ws.H = carve<double2>(cp, NL2);
    ws.H2 = carve<double2>(cp, NL2);
    ws.Y = carve<double2>(cp, NL2);
    ws.Ysort = carve<double2>(cp, NL2);
    ws.order = carve<int32_t>(cp, NL);
    ws.evals = carve<double>(cp, NL);
    ws.conv = carve<int32_t>(cp, 4);
    ws.acc = carve<double>(cp, 2);
    ws.W = carve<double2>(cp, NL2);
    ws.C = carve<double2>(cp, NL2);
    ws.bar = carve<unsigned int>(cp, 4);
    ws.jacc = carve<double>(cp, 2 * 4096);
    ws.Q1 = carve<double2>(cp, (size_t)n * NL);
    ws.Ytmp = carve<double2>(cp, (size_t)n * NL);
    ws.gws_elems = std::max<size_t>(NL2 * 4, (size_t)8 << 20);
    ws.gws = carve<double2>(cp, ws.gws_elems);
    ws.ows_bytes = ozaki_ws_bytes(NL, n);
    ws.ows = carve<char>(cp, ws.ows_bytes);
    ws.Qall = carve<double2>(cp, (size_t)n * NL);
    ws.P = carve<double2>(cp, (size_t)std::max(terms, RSRR_MAX_TERMS) * NL2);
    ws.end = cp;
}

static size_t ws_bytes(int NL, int64_t n, int terms) {
    ProjWs ws;
    char *base = reinterpret_cast<char *>((uintptr_t)0);
    carve_ws(base, ws, NL, n, terms);
    return (size_t)(ws.end - base);
}

size_t projection_ws_bytes(int NL, int64_t n, int terms) { return ws_bytes(NL, n, terms); }

// Orthonormal basis of the dominant singular subspace of Sn = X D^{-1}:
// deflated multi-level Gram.  Level l works on the remainder R_l (R_0 = Sn):
//   G_l = R_l^H R_l; pivoted Cholesky G_l ~ B B^H stopped when the largest
//   remaining diagonal is <= max(lev_tol^2 * maxdiag(G_l), floor^2 sigma_1^2)
//   (lev_tol = 1e-6: the kept directions sit far above the Gram's rounding);
//   B^H B = Y Lambda Y^H (Jacobi); new directions R_l B Y Lambda^{-1} for the
//   eigenvalues well above the level's threshold, orthogonalised twice
//   against the basis so far and once more within the block (Jacobi on its
//   Gram); then R_{l+1} = R_l - Qall Qall^H R_l, twice.
// Each level sees only directions far above its own rounding level, so the
// levels together resolve singular values down to ~lev_tol^L of sigma_1.
rsrr_status Handle::project(cudaStream_t s) {
    using cplx = std::complex<double>;
    const int NL = N * L;
    const int64_t nn = n;
    if (opts.method == RSRR_METHOD_SS_RI) return RSRR_OK;  // SS-RI works on the samples directly
    // columns of the matrix whose basis is taken: S (N L) or the moments M (K L)
    const int nc = opts.method == RSRR_METHOD_SSRR_M ? opts.K * L : NL;
    if (!proj_ws) {
        const size_t bytes = ws_bytes(NL, nn, m);
        void *p = nullptr;
        cudaError_t e = raw_alloc(&p, bytes);
        if (e != cudaSuccess) return fail(RSRR_ENOMEM, "projection work space", e);
        proj_ws = p;
        proj_ws_bytes = bytes;
    }
    ProjWs ws;
    carve_ws(reinterpret_cast<char *>(proj_ws), ws, NL, nn, m);
    d_Q = ws.Qall;
    d_P = ws.P;
    Gemm gm;
    gm.ws = ws.gws;
    gm.ws_elems = ws.gws_elems;
    gm.counter = &launches;
    gm.method = opts.gemm;
    gm.ows = ws.ows;
    gm.ows_bytes = ws.ows_bytes;
    gm.tmo = d_tmo;
    if (opts.timing) {
        gm.timer = this;
        gemm_pool.used = 0;
        tc_pool.used = 0;
        gemm_flops = 0.0;
        tc_flops = 0.0;
        gemm_timed = true;
    }
    rsrr_status mst = mark(6, s);
    if (mst != RSRR_OK) return mst;

    const double2 *src = d_X;
    if (opts.method == RSRR_METHOD_SSRR_M) {
        // M = [M_0 ... M_{K-1}], M_a = sum_i w_i s_i^a X_i (Eq. 40, Eq. 48): for
        // every probe column l, M(:, a L + l) = sum_i X(:, i L + l) C(i, a), one
        // product of the strided columns of S by C (N x K) in ws.W
        std::vector<cplx> w;
        moment_weights(w);
        const double rho = std::max(region.a, region.b);
        const cplx gamma(region.center.re, region.center.im);
        const int K = opts.K;
        std::vector<double2> Cm((size_t)N * K);
        for (int i = 0; i < N; ++i) {
            const cplx si = (z[i] - gamma) / rho;
            cplx pw = 1.0;
            for (int a = 0; a < K; ++a) {
                const cplx c = w[i] * pw;
                Cm[(size_t)a * N + i] = make_double2(c.real(), c.imag());
                pw *= si;
            }
        }
        PK(cudaMemcpyAsync(ws.W, Cm.data(), sizeof(double2) * Cm.size(), cudaMemcpyHostToDevice, s), "moment coefs");
        for (int l = 0; l < L; ++l)
            PK(gm.run((int)nn, K, N, false, d_X + (size_t)l * nn, (int64_t)L * nn, ws.W, N, ws.Ytmp + (size_t)l * nn,
                      (int64_t)L * nn, s), "M = S Z");
        PK(cudaStreamSynchronize(s), "moment coefs");  // the host copy of the coefficients stays valid until here
        src = ws.Ytmp;
    }
    // (A8) unit-norm columns: R_0 = X D^{-1} (or M D^{-1})
    colnorm_kernel<<<nc, 256, 0, s>>>(ws.norms, src, nn);
    scale_cols_kernel<<<grid1d(nn * nc), 256, 0, s>>>(ws.Q1, src, ws.norms, nn, nc);
    PK(cudaGetLastError(), "normalise");
    launches += 2;
    double2 *R = ws.Q1;
    const double lev_tol = 1e-6;
    // resolution floor of the basis: the caller's, or automatic -- the samples'
    // own accuracy (a tenth of eta_tol for the refined mixed-precision samples,
    // 1e-12 for the FP64 path): singular values of S below it are noise of the
    // samples, and keeping them only grows k (and the k^3 SS-FULL behind it).
    // The moment matrix of SSRR-M is not S: its higher moments carry the
    // eigen-directions scaled by ((lambda - gamma) / rho)^a, far below its
    // sigma_1, so it keeps the fixed 1e-12.
    const double floor_auto =
        opts.precision == RSRR_PREC_MIXED && opts.method == RSRR_METHOD_RSRR ? 0.1 * opts.eta_tol : 1e-12;
    const double floor_ = std::max(opts.delta, opts.delta_floor > 0.0 ? opts.delta_floor : floor_auto);
    int kt = 0;            // columns of Qall so far
    double s1sq = 0.0;     // sigma_1^2 of Sn (from level 0)
    double smallest = 0.0; // smallest kept eigenvalue (for sigma_k)
    kc = 0;
    for (int lev = 0; lev < 6 && kt < nc; ++lev) {
        // (A9) Gram of the remainder and its largest diagonal
        double maxd = 1.0;
        PK(gm.run(nc, nc, (int)nn, true, R, nn, R, nn, ws.G, nc, s, true), "Gram");
        max_diag_kernel<<<1, 256, 0, s>>>(ws.acc, ws.G, nc);
        PK(cudaMemcpyAsync(&maxd, ws.acc, sizeof(double), cudaMemcpyDeviceToHost, s), "maxdiag");
        PK(cudaStreamSynchronize(s), "maxdiag sync");
        launches += 1;
        const double tau = std::max(lev_tol * lev_tol * maxd, floor_ * floor_ * s1sq);
        PK(cudaMemsetAsync(ws.state, 0, sizeof(int32_t) * 4, s), "memset");
        PK(cudaMemsetAsync(ws.bar, 0, sizeof(unsigned int) * 4, s), "memset");
        diag_real_kernel<<<(nc + 255) / 256, 256, 0, s>>>(ws.dbuf, ws.G, nc);
        PK(launch_coop(pchol_persistent_kernel, (nc + 255) / 256, s, (const double2 *)ws.G, nc,
                       ws.Lm, ws.dbuf, tau, ws.state, ws.bar, (int32_t *)nullptr), "pivoted Cholesky");
        launches += 2;
        int32_t st2[2];
        unsigned int bar_err = 0;
        PK(cudaMemcpyAsync(st2, ws.state, sizeof st2, cudaMemcpyDeviceToHost, s), "kc");
        PK(cudaMemcpyAsync(&bar_err, ws.bar + 2, sizeof bar_err, cudaMemcpyDeviceToHost, s), "kc");
        PK(cudaStreamSynchronize(s), "kc sync");
        if (bar_err) return fail(RSRR_ETIMEOUT, "rsrr_project: grid barrier timeout (pivoted Cholesky)");
        const int kcl = st2[0] ? st2[1] : nc;
        if (kcl < 1) break;
        kc += kcl;
        // small Hermitian eigenproblem B^H B
        PK(gm.run(kcl, kcl, nc, true, ws.Lm, nc, ws.Lm, nc, ws.H, kcl, s, true), "B^H B");
        PK(jacobi_eig(ws, kcl, s, &launches), "Jacobi (B^H B)");
        std::vector<double> ev(kcl);
        PK(cudaMemcpyAsync(ev.data(), ws.evals, sizeof(double) * kcl, cudaMemcpyDeviceToHost, s), "evals");
        PK(cudaMemcpyAsync(&bar_err, ws.bar + 2, sizeof bar_err, cudaMemcpyDeviceToHost, s), "evals");
        PK(cudaStreamSynchronize(s), "evals sync");
        if (bar_err) return fail(RSRR_ETIMEOUT, "rsrr_project: grid barrier timeout (Jacobi)");
        if (lev == 0) s1sq = std::max(ev[0], 0.0);
        const double keep_tol = std::max(1e-2 * tau, floor_ * floor_ * s1sq);
        int kb = 0;
        for (int j = 0; j < kcl; ++j)
            if (ev[j] > keep_tol) kb = j + 1;
        if (kb < 1) break;
        smallest = ev[kb - 1];
        if (kt + kb > nc) kb = nc - kt;
        // new directions Qb = R B Y_kb Lambda_kb^{-1} (n x kb) into Ytmp
        PK(gm.run(nc, kb, kcl, false, ws.Lm, nc, ws.Ysort, kcl, ws.W, nc, s), "B Y");
        scale_rc_kernel<<<grid1d((int64_t)nc * kb), 256, 0, s>>>(ws.W, nc, nc, kb, nullptr,
                                                                 ws.evals, false, false);
        launches += 1;
        PK(gm.run((int)nn, kb, nc, false, R, nn, ws.W, nc, ws.Ytmp, nn, s), "R W");
        // orthogonalise against the basis so far, twice
        for (int pass = 0; pass < 2 && kt > 0; ++pass) {
            PK(gm.run(kt, kb, (int)nn, true, ws.Qall, nn, ws.Ytmp, nn, ws.C, kt, s), "Q^H Qb");
            PK(gm.run((int)nn, kb, kt, false, ws.Qall, nn, ws.C, kt, ws.Ytmp, nn, s, false, -1.0, 1.0),
               "Qb -= Q C");
        }
        // within the block: Cholesky QR with column pivoting, Qb^H Qb =
        // P T T^H P^T, stopped at 1e-10 of the largest diagonal; Qall(:, kt:
        // kt+kb2) = Qb S T^{-H} (a cyclic Jacobi on this nearly-identity Gram,
        // with its clustered eigenvalues, took 18 sweeps where the one on
        // B^H B takes 7)
        PK(gm.run(kb, kb, (int)nn, true, ws.Ytmp, nn, ws.Ytmp, nn, ws.H, kb, s, true), "Qb^H Qb");
        double maxd2 = 0.0;
        int kb2 = 0;
        max_diag_kernel<<<1, 256, 0, s>>>(ws.acc, ws.H, kb);
        diag_real_kernel<<<(kb + 255) / 256, 256, 0, s>>>(ws.dbuf, ws.H, kb);
        launches += 2;
        PK(cudaMemcpyAsync(&maxd2, ws.acc, sizeof(double), cudaMemcpyDeviceToHost, s), "block Gram diagonal");
        PK(cudaStreamSynchronize(s), "block Gram diagonal");
        PK(cudaMemsetAsync(ws.state, 0, sizeof(int32_t) * 4, s), "memset");
        PK(cudaMemsetAsync(ws.bar, 0, sizeof(unsigned int) * 4, s), "memset");
        PK(launch_coop(pchol_persistent_kernel, (kb + 255) / 256, s, (const double2 *)ws.H, kb, ws.Lm, ws.dbuf,
                       1e-10 * maxd2, ws.state, ws.bar, ws.order), "pivoted Cholesky (Qb^H Qb)");
        launches += 1;
        {
            int32_t st3[2];
            PK(cudaMemcpyAsync(st3, ws.state, sizeof st3, cudaMemcpyDeviceToHost, s), "block rank");
            PK(cudaMemcpyAsync(&bar_err, ws.bar + 2, sizeof bar_err, cudaMemcpyDeviceToHost, s), "block rank");
            PK(cudaStreamSynchronize(s), "block rank sync");
            if (bar_err) return fail(RSRR_ETIMEOUT, "rsrr_project: grid barrier timeout (pivoted Cholesky)");
            kb2 = st3[0] ? st3[1] : kb;
        }
        if (kb2 < 1) break;
        tri_from_pchol_kernel<<<grid1d((int64_t)kb2 * kb2), 256, 0, s>>>(ws.H2, ws.Lm, ws.order, kb, kb2);
        tri_inverse_lower_kernel<<<(kb2 + 7) / 8, 256, 0, s>>>(ws.Y, ws.H2, kb2);
        PK(cudaMemsetAsync(ws.Ysort, 0, sizeof(double2) * (size_t)kb * kb2, s), "memset");
        scatter_inverse_fill_kernel<<<grid1d((int64_t)kb2 * kb2), 256, 0, s>>>(ws.Ysort, ws.Y, ws.order, kb, kb2);
        PK(cudaGetLastError(), "block Cholesky QR");
        launches += 3;
        double2 *Qnew = ws.Qall + (size_t)kt * nn;
        PK(gm.run((int)nn, kb2, kb, false, ws.Ytmp, nn, ws.Ysort, kb, Qnew, nn, s), "Qb S T^-H");
        const int kprev = kt;
        kt += kb2;
        // deflate the remainder: pass 1 against the new block (R is already
        // orthogonal to the earlier blocks), pass 2 against the whole basis.
        // Before pass 1's update, the column norms the deflation would leave,
        // diag(G) - |Qnew^H R|^2, tell whether another level is needed; if
        // not, R is not needed any more and the updates are skipped.
        PK(gm.run(kb2, nc, (int)nn, true, Qnew, nn, R, nn, ws.C, kb2, s), "Qnew^H R");
        remainder_norm_kernel<<<(nc + 255) / 256, 256, 0, s>>>(ws.dbuf, ws.G, ws.C, kb2, nc);
        max_vec_kernel<<<1, 256, 0, s>>>(ws.acc, ws.dbuf, nc);
        launches += 2;
        double rem = 0.0;
        PK(cudaMemcpyAsync(&rem, ws.acc, sizeof(double), cudaMemcpyDeviceToHost, s), "remainder");
        PK(cudaStreamSynchronize(s), "remainder sync");
        if (!(rem > floor_ * floor_ * s1sq) || kt >= nc) break;
        PK(gm.run((int)nn, nc, kb2, false, Qnew, nn, ws.C, kb2, R, nn, s, false, -1.0, 1.0),
           "R -= Qnew C");
        PK(gm.run(kt, nc, (int)nn, true, ws.Qall, nn, R, nn, ws.C, kt, s), "Q^H R");
        PK(gm.run((int)nn, nc, kt, false, ws.Qall, nn, ws.C, kt, R, nn, s, false, -1.0, 1.0),
           "R -= Q C");
        (void)kprev;
    }
    if (kt < 1) return fail(RSRR_ESTATE, "rsrr_project: empty basis");
    k = kt;
    sigma1 = std::sqrt(s1sq);
    sigmak = std::sqrt(std::max(smallest, 0.0));

    // (A10) P_q = Q^H (A_q Q); for the dense kernel the A_p are the Taylor
    // coefficients about the region centre, generated in place one after the
    // other in the (now free) complex128 matrix storage of the first point
    if (dense_terms) {  // caller-supplied dense A_q, resident on the device
        for (int q = 0; q < m; ++q) {
            const double2 *Aq = d_Aterms + (size_t)q * nn * nn;
            PK(gm.run((int)nn, k, (int)nn, false, Aq, nn, d_Q, nn, ws.Ytmp, nn, s), "A_q Q");
            PK(gm.run(k, k, (int)nn, true, d_Q, nn, ws.Ytmp, nn, d_P + (size_t)q * k * k, k, s), "Q^H A_q Q");
        }
    } else if (dense) {
        const double2 c = make_double2(region.center.re, region.center.im);
        for (int q = 0; q < m; ++q) {
            PK(launch_taylor_step(d_T64, d_points, c, diag, (int)nn, q, s), "Taylor coefficient");
            PK(gm.run((int)nn, k, (int)nn, false, d_T64, nn, d_Q, nn, ws.Ytmp, nn, s), "A_p Q");
            PK(gm.run(k, k, (int)nn, true, d_Q, nn, ws.Ytmp, nn, d_P + (size_t)q * k * k, k, s), "Q^H A_p Q");
            launches += 1;
        }
    }
    for (int q = 0; q < m && !dense; ++q) {
        dim3 grid((unsigned)((nn + 127) / 128), k);
        spmm_kernel<<<grid, 128, 0, s>>>(ws.Ytmp, d_Q, d_row_ptr, d_col_idx, d_vals + (size_t)q * nnz,
                                         (int)nn, k);
        PK(cudaGetLastError(), "SpMM");
        PK(gm.run(k, k, (int)nn, true, d_Q, nn, ws.Ytmp, nn, d_P + (size_t)q * k * k, k, s), "Q^H A Q");
        launches += 1;
    }
    mst = mark(7, s);
    if (mst != RSRR_OK) return mst;
    timed_project = opts.timing != 0;
    return RSRR_OK;
}

}  // namespace rsrr

using rsrr::Handle;

extern "C" {

rsrr_status rsrr_project(rsrr_t *hh, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return RSRR_EINVAL;
    if (!h->sampled) return h->fail(RSRR_ESTATE, "rsrr_project: no rsrr_sample yet");
    rsrr_status st = h->project((cudaStream_t)stream);
    h->projected = (st == RSRR_OK);
    return st;
}

rsrr_status rsrr_get_Q(rsrr_t *hh, rsrr_c128 *dst, int32_t dst_on_device, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !dst) return RSRR_EINVAL;
    if (!h->projected || !h->d_Q) return h->fail(RSRR_ESTATE, "rsrr_get_Q: no basis (rsrr_project, RSRR or SSRR-M)");
    const size_t bytes = sizeof(double2) * (size_t)h->n * h->k;
    cudaError_t e;
    if (dst_on_device) {
        e = cudaMemcpyAsync(dst, h->d_Q, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    } else {
        e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaMemcpy(dst, h->d_Q, bytes, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return h->fail(RSRR_ECUDA, "rsrr_get_Q", e);
    return RSRR_OK;
}

rsrr_status rsrr_get_projected(rsrr_t *hh, rsrr_c128 *dst, int32_t dst_on_device, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !dst) return RSRR_EINVAL;
    if (!h->projected || !h->d_P) return h->fail(RSRR_ESTATE, "rsrr_get_projected: no rsrr_project yet");
    const size_t bytes = sizeof(double2) * (size_t)h->m * h->k * h->k;
    cudaError_t e;
    if (dst_on_device) {
        e = cudaMemcpyAsync(dst, h->d_P, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    } else {
        e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaMemcpy(dst, h->d_P, bytes, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return h->fail(RSRR_ECUDA, "rsrr_get_projected", e);
    return RSRR_OK;
}

}  // extern "C"

// ==========================================================================
// rsrr_solve: SS-FULL on the host, v = Q g and residuals on the GPU
// ==========================================================================
#include "ssfull_host.h"

namespace rsrr {

// rr[c] = ||T(lam_c) v_c||^2, vv[c] = ||v_c||^2 (FP64, CSR, coefficients per pair)
__global__ void eig_residual_kernel(const double2 *__restrict__ V, const double2 *__restrict__ coef,
                                    const int32_t *__restrict__ row_ptr,
                                    const int32_t *__restrict__ col_idx,
                                    const double *__restrict__ vals, int64_t nnz, int m, int n,
                                    double *__restrict__ rr, double *__restrict__ vv) {
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0, v2 = 0.0;
    if (i < n) {
        double2 s = make_double2(0.0, 0.0);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            double2 a = make_double2(0.0, 0.0);
            for (int q = 0; q < m; ++q) {
                const double v = vals[(int64_t)q * nnz + e];
                a.x = fma(coef[c * m + q].x, v, a.x);
                a.y = fma(coef[c * m + q].y, v, a.y);
            }
            s = cfma(s, a, V[(int64_t)c * n + col_idx[e]]);
        }
        r2 = s.x * s.x + s.y * s.y;
        const double2 x = V[(int64_t)c * n + i];
        v2 = x.x * x.x + x.y * x.y;
    }
    for (int off = 16; off; off >>= 1) {
        r2 += shfl_down(r2, off);
        v2 += shfl_down(v2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(rr + c, r2);
        atomicAdd(vv + c, v2);
    }
}

// SS-RI (Section 3.3) on the resident samples: F(z_i) = U^H X_i (Eq. 14) by
// one product on the GPU, the moments A_a = sum_i w_i s_i^a F(z_i), a < 2K
// (Eq. 18, scaled powers s_i = (z_i - gamma)/rho) on the host, the Hankel
// pencil, truncated SVD and gap test, eigenpairs of A (Eq. 33-38) by the
// SS-FULL finish, and the eigenvector coefficients in the sample space:
// v = M W0 Sigma0^{-1} b = S ZWB with ZWB((i, l), c) = sum_a w_i s_i^a
// (W0 Sigma0^{-1} B)((a, l), c) (Eq. 39-41).
rsrr_status Handle::ss_ri(cudaStream_t s, std::vector<std::complex<double>> &lam,
                          std::vector<std::complex<double>> &ZWB, int &nbar, double &gmax) {
    using cplx = std::complex<double>;
    const int NL = N * L, K = opts.K;
    if (!proj_ws) {
        const size_t bytes = ws_bytes(NL, n, m);
        void *p = nullptr;
        cudaError_t e = raw_alloc(&p, bytes);
        if (e != cudaSuccess) return fail(RSRR_ENOMEM, "SS-RI work space", e);
        proj_ws = p;
        proj_ws_bytes = bytes;
    }
    ProjWs ws;
    carve_ws(reinterpret_cast<char *>(proj_ws), ws, NL, n, m);
    Gemm gm;
    gm.ws = ws.gws;
    gm.ws_elems = ws.gws_elems;
    gm.counter = &launches;
    gm.method = opts.gemm;
    gm.ows = ws.ows;
    gm.ows_bytes = ws.ows_bytes;
    gm.tmo = d_tmo;
    PK(gm.run(L, NL, (int)n, true, d_U, n, d_X, n, ws.W, L, s), "U^H S");
    std::vector<double2> Y((size_t)L * NL);
    PK(cudaMemcpyAsync(Y.data(), ws.W, sizeof(double2) * Y.size(), cudaMemcpyDeviceToHost, s), "U^H S");
    PK(cudaStreamSynchronize(s), "U^H S");
    std::vector<cplx> w;
    moment_weights(w);
    const double rho = std::max(region.a, region.b);
    const cplx gamma(region.center.re, region.center.im);
    std::vector<std::vector<cplx>> Am(2 * K, std::vector<cplx>((size_t)L * L, 0.0));
    std::vector<cplx> sp((size_t)N * 2 * K);  // w_i s_i^a
    for (int i = 0; i < N; ++i) {
        const cplx si = (z[i] - gamma) / rho;
        cplx pw = 1.0;
        for (int a = 0; a < 2 * K; ++a) {
            sp[(size_t)i * 2 * K + a] = w[i] * pw;
            pw *= si;
        }
    }
    for (int a = 0; a < 2 * K; ++a)
        for (int i = 0; i < N; ++i) {
            const cplx c = sp[(size_t)i * 2 * K + a];
            for (int cc = 0; cc < L; ++cc)
                for (int r = 0; r < L; ++r) {
                    const double2 y = Y[((size_t)i * L + cc) * L + r];
                    Am[a][(size_t)cc * L + r] += c * cplx(y.x, y.y);
                }
        }
    std::vector<cplx> Gdummy, WB;
    if (ss_full_finish(Am, L, K, gamma, rho, opts.host_threads, lam, Gdummy, nbar, gmax, &WB) != 0)
        return fail(RSRR_ESINGULAR, "rsrr_solve: the SS-RI moments vanish");
    ZWB.assign((size_t)NL * nbar, 0.0);
    for (int c = 0; c < nbar; ++c)
        for (int i = 0; i < N; ++i)
            for (int l = 0; l < L; ++l) {
                cplx acc = 0.0;
                for (int a = 0; a < K; ++a) acc += sp[(size_t)i * 2 * K + a] * WB[(size_t)c * K * L + a * L + l];
                ZWB[(size_t)c * NL + (size_t)i * L + l] = acc;
            }
    return RSRR_OK;
}

rsrr_status Handle::solve(rsrr_result *out) {
    using cplx = std::complex<double>;
    cudaStream_t s = hs;
    PK(wait(), "solve sync");
    {  // a bounded wait of one of this handle's tensor-core products that ran
       // out since rsrr_sample (the handle's own status word, read on its stream)
        unsigned int tmo = 0;
        PK(cudaMemcpyAsync(&tmo, d_tmo, sizeof tmo, cudaMemcpyDeviceToHost, s), "status word");
        PK(cudaStreamSynchronize(s), "status word");
        if (tmo != 0)
            return fail(RSRR_ETIMEOUT, "rsrr_solve: a bounded tensor-core wait ran out in sample or project");
    }
    const auto D2H = cudaMemcpyDeviceToHost;
    const auto H2D = cudaMemcpyHostToDevice;
    std::vector<cplx> lam, G;
    int nbar = 0;
    double gmax = 0.0;
    const cplx gamma(region.center.re, region.center.im);
    const int NL = N * L;
    // the eigenvectors are v = B g: B = Q (k columns) for the projected
    // methods, B = S (N L columns) for SS-RI
    const double2 *Bsrc = d_Q;
    int kb = k;
    if (opts.method == RSRR_METHOD_SS_RI) {
        const rsrr_status rst = ss_ri(s, lam, G, nbar, gmax);
        if (rst != RSRR_OK) return rst;
        Bsrc = d_X;
        kb = NL;
    } else {
        // moments of T_Q^{-1} on the GPU, the rest of SS-FULL on the host; f of
        // every held term at the contour nodes (the N_Q trapezoid nodes of
        // Eq. 58, or composite Gauss on a rectangle)
        std::vector<cplx> zq, wq, fq;
        contour_quadrature(opts.NQ, zq, wq);
        rsrr_status est = eval_terms(zq.data(), (int64_t)zq.size(), fq);
        if (est != RSRR_OK) return est;
        std::vector<std::vector<cplx>> Am;
        const rsrr_status mst = ssfull_moments(fq, zq, wq, opts.KQ, Am);
        if (mst != RSRR_OK) return mst;
        if (ss_full_finish(Am, k, opts.KQ, gamma, std::max(region.a, region.b), opts.host_threads, lam, G,
                           nbar, gmax) != 0)
            return fail(RSRR_ESINGULAR, "rsrr_solve: the SS-FULL moments vanish");
    }
    // v = B g on the GPU
    ProjWs ws;
    carve_ws(reinterpret_cast<char *>(proj_ws), ws, NL, n, m);
    Gemm gm;
    gm.ws = ws.gws;
    gm.ws_elems = ws.gws_elems;
    gm.counter = &launches;
    // G (k x nbar), V = Q G (n x nbar), f_i(lam_c) and the residual sums in a
    // buffer of their own (nbar may exceed the sample count)
    const size_t gbytes = sizeof(double2) * (size_t)kb * nbar;
    const size_t vbytes = sizeof(double2) * (size_t)n * nbar;
    const size_t cbytes = sizeof(double2) * (size_t)nbar * std::max(m, 2);
    void *buf = nullptr;
    // dense terms: A_i V and the accumulated T(lambda) V as well
    const size_t ybytes = dense_terms ? 2 * vbytes : 0;
    const size_t tbytes = gbytes + vbytes + cbytes + sizeof(double) * 2 * nbar + ybytes;
    PK(pool ? cudaMallocFromPoolAsync(&buf, tbytes, pool, s) : cudaMalloc(&buf, tbytes), "solve buffers");
    struct Free {
        Handle *h;
        void *p;
        ~Free() { h->raw_free(p); }
    } guard{this, buf};
    double2 *d_G = reinterpret_cast<double2 *>(buf);
    double2 *d_V = reinterpret_cast<double2 *>(reinterpret_cast<char *>(buf) + gbytes);
    double2 *d_cf = reinterpret_cast<double2 *>(reinterpret_cast<char *>(buf) + gbytes + vbytes);
    double *d_rr = reinterpret_cast<double *>(reinterpret_cast<char *>(buf) + gbytes + vbytes + cbytes);
    double *d_vv = d_rr + nbar;
    PK(cudaMemcpyAsync(d_G, G.data(), gbytes, H2D, s), "G");
    PK(gm.run((int)n, nbar, kb, false, Bsrc, n, d_G, kb, d_V, n, s), "B G");
    std::vector<double> t1(nbar, 0.0);
    // f of every held term at the eigenvalues (residual scale, sparse and dense-terms kinds)
    std::vector<cplx> flam;
    if (!dense || dense_terms) {
        rsrr_status fst = eval_terms(lam.data(), nbar, flam);
        if (fst != RSRR_OK) return fst;
    }
    if (dense_terms) {
        std::vector<double2> cf((size_t)nbar * m);
        for (size_t e = 0; e < cf.size(); ++e) cf[e] = make_double2(flam[e].real(), flam[e].imag());
        PK(cudaMemcpyAsync(d_cf, cf.data(), sizeof(double2) * cf.size(), H2D, s), "coef");
        double2 *d_Y = reinterpret_cast<double2 *>(reinterpret_cast<char *>(d_rr) + sizeof(double) * 2 * nbar);
        double2 *d_TV = d_Y + (size_t)n * nbar;
        // T(lambda_c) v_c = sum_i f_i(lambda_c) (A_i V)(:, c)
        for (int i = 0; i < m; ++i) {
            PK(gm.run((int)n, nbar, (int)n, false, d_Aterms + (size_t)i * n * n, n, d_V, n, d_Y, n, s), "A_i V");
            PK(launch_accum_term_cols(d_TV, d_Y, d_cf, m, i, (int)n, nbar, i == 0, s), "T V");
            launches += 1;
        }
        PK(launch_col_norms2(d_TV, d_V, (int)n, nbar, d_rr, d_vv, s), "residual norms");
        launches += 1;
    } else if (dense) {
        std::vector<double2> lz(nbar);
        for (int c = 0; c < nbar; ++c) lz[c] = make_double2(lam[c].real(), lam[c].imag());
        PK(cudaMemcpyAsync(d_cf, lz.data(), sizeof(double2) * nbar, H2D, s), "lam");
        PK(cudaMemsetAsync(d_rr, 0, sizeof(double) * 2 * nbar, s), "memset");
        double *d_t1 = reinterpret_cast<double *>(d_cf + nbar);
        PK(cudaMemsetAsync(d_t1, 0, sizeof(double) * nbar, s), "memset");
        PK(launch_dense_eig_residual(d_V, d_cf, d_points, diag, (int)n, nbar, d_rr, d_vv, d_t1, s),
           "dense eig residual");
        PK(cudaMemcpyAsync(t1.data(), d_t1, sizeof(double) * nbar, D2H, s), "t1");
        launches += 1;
    } else {
        std::vector<double2> cf((size_t)nbar * m);
        for (size_t e = 0; e < cf.size(); ++e) cf[e] = make_double2(flam[e].real(), flam[e].imag());
        PK(cudaMemcpyAsync(d_cf, cf.data(), sizeof(double2) * cf.size(), H2D, s), "coef");
        PK(cudaMemsetAsync(d_rr, 0, sizeof(double) * 2 * nbar, s), "memset");
        eig_residual_kernel<<<dim3((unsigned)((n + 255) / 256), nbar), 256, 0, s>>>(
            d_V, d_cf, d_row_ptr, d_col_idx, d_vals, nnz, m, (int)n, d_rr, d_vv);
        PK(cudaGetLastError(), "eig residual");
        launches += 1;
    }
    std::vector<double> rr(nbar), vv(nbar);
    std::vector<cplx> V((size_t)n * nbar);
    PK(cudaMemcpyAsync(rr.data(), d_rr, sizeof(double) * nbar, D2H, s), "rr");
    PK(cudaMemcpyAsync(vv.data(), d_vv, sizeof(double) * nbar, D2H, s), "vv");
    PK(cudaMemcpyAsync(V.data(), d_V, sizeof(double2) * V.size(), D2H, s), "V");
    PK(cudaStreamSynchronize(s), "solve results");
    struct Pair { cplx lam; double res; int c; };
    std::vector<Pair> keep;
    for (int c = 0; c < nbar; ++c) {
        if (!inside(lam[c])) continue;
        double scale = 0.0;
        if (dense && !dense_terms) scale = t1[c];  // ||T(lam)||_1 of the kernel computed directly
        else scale = residual_scale(flam.data() + (size_t)c * m);  // sum_u |f_u(lam)| ||A_u||_1
        const double res = std::sqrt(rr[c]) / (scale * std::sqrt(vv[c]));
        if (!(res <= opts.res_tol)) continue;
        keep.push_back({lam[c], res, c});
    }
    std::sort(keep.begin(), keep.end(), [](const Pair &a, const Pair &b) {
        if (std::abs(a.lam) != std::abs(b.lam)) return std::abs(a.lam) < std::abs(b.lam);
        return std::arg(a.lam) < std::arg(b.lam);
    });
    res_lam.resize(keep.size());
    res_res.resize(keep.size());
    res_V.resize((size_t)n * keep.size());
    for (size_t t = 0; t < keep.size(); ++t) {
        res_lam[t] = {keep[t].lam.real(), keep[t].lam.imag()};
        res_res[t] = keep[t].res;
        const double nv = std::sqrt(vv[keep[t].c]);
        for (int64_t i = 0; i < n; ++i) {
            const cplx v = V[(size_t)keep[t].c * n + i] / nv;
            res_V[t * n + i] = {v.real(), v.imag()};
        }
    }
    out->count = (int32_t)keep.size();
    out->nbar = nbar;
    out->gmax = gmax;
    out->lam = res_lam.data();
    out->res = res_res.data();
    out->V = res_V.data();
    return gmax >= opts.tol_gap ? RSRR_OK : RSRR_WGAP;
}

}  // namespace rsrr

extern "C" rsrr_status rsrr_solve(rsrr_t *hh, rsrr_result *out) {
    rsrr::Handle *h = reinterpret_cast<rsrr::Handle *>(hh);
    if (!h || !out) return RSRR_EINVAL;
    if (h->opts.method == RSRR_METHOD_SS_RI ? !h->sampled : !h->projected)
        return h->fail(RSRR_ESTATE, "rsrr_solve: no rsrr_project (rsrr_sample for SS-RI) yet");
    const rsrr_status st = h->solve(out);
    h->solved = st >= 0;
    return st;
}
