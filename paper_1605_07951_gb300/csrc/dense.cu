// Resolvent sampling on dense BEM-like T(z_j) (RSRR step 2, Section 4.3, for
// the Nystrom single-layer kernel of Section 2.1):
//   T(z)_ij = exp(i z r_ij) / (4 pi r_ij) (i != j), T_ii = diag,
// assembled per sampling point, factored by a batched blocked LU with partial
// pivoting, solved for the L probe columns with the block inverses of the
// factorisation, and refined with FP64 residuals (the GEMM of proj.cu).
//
// Dense storage of one point: column major n x n (lda = n).  Pivoting is
// applied dense-style inside an NB-column block and to the trailing columns,
// never to the columns already factored: the solve applies each block's
// interchanges just before that block's elimination, as the band solve does.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

constexpr double kFourPi = 12.566370614359172;

RSRR_DEV void store_d(float2 *p, double2 v) { *p = to_c64(v); }
RSRR_DEV void store_d(double2 *p, double2 v) { *p = v; }

// ---------------------------------------------------------------- assembly
// complex64 entries from FP32 sincos/exp (the factor is complex64 anyway);
// complex128 entries in FP64 (used by the FP64 residual and the FP64 path).
__global__ void assemble_dense_c64_kernel(float2 *__restrict__ A_all, const double *__restrict__ pts,
                                          const double2 *__restrict__ zs, double diag, int n) {
    const int pt = blockIdx.y;
    const float zr = (float)zs[pt].x, zi = (float)zs[pt].y;
    float2 *A = A_all + (size_t)pt * n * n;
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / n), i = (int)(q - (int64_t)j * n);
        float2 v;
        if (i == j) {
            v = make_float2((float)diag, 0.f);
        } else {
            const float dx = (float)(pts[3 * i] - pts[3 * j]), dy = (float)(pts[3 * i + 1] - pts[3 * j + 1]),
                        dz = (float)(pts[3 * i + 2] - pts[3 * j + 2]);
            const float r = sqrtf(dx * dx + dy * dy + dz * dz);
            const float mag = expf(-zi * r) / ((float)kFourPi * r);
            float s, c;
            sincosf(zr * r, &s, &c);
            v = make_float2(mag * c, mag * s);
        }
        A[q] = v;
    }
}

__global__ void assemble_dense_c128_kernel(double2 *__restrict__ A_all, const double *__restrict__ pts,
                                           const double2 *__restrict__ zs, double diag, int n) {
    const int pt = blockIdx.y;
    const double zr = zs[pt].x, zi = zs[pt].y;
    double2 *A = A_all + (size_t)pt * n * n;
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / n), i = (int)(q - (int64_t)j * n);
        double2 v;
        if (i == j) {
            v = make_double2(diag, 0.0);
        } else {
            const double dx = pts[3 * i] - pts[3 * j], dy = pts[3 * i + 1] - pts[3 * j + 1],
                         dz = pts[3 * i + 2] - pts[3 * j + 2];
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            const double mag = exp(-zi * r) / (kFourPi * r);
            double s, c;
            sincos(zr * r, &s, &c);
            v = make_double2(mag * c, mag * s);
        }
        A[q] = v;
    }
}

// T(z_j) = sum_i f_i(z_j) A_i for caller-supplied dense A_i (m x n^2
// complex128, term-major): every thread loads the m coefficients of one
// entry once and writes that entry of every point of the chunk, so the A_i
// are read once per chunk of points and the N matrices written once (the
// write stream is the bound).  coef is point-major, f_i(z_j) at [j m + i].
__global__ void assemble_dense_terms_kernel(double2 *__restrict__ T_all, const double2 *__restrict__ A,
                                            const double2 *__restrict__ coef, int64_t nn2, int j0, int nj,
                                            int m) {
    extern __shared__ double2 s_cf[];  // nj x m
    for (int t = threadIdx.x; t < nj * m; t += blockDim.x) s_cf[t] = coef[(size_t)j0 * m + t];
    __syncthreads();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nn2;
         q += (int64_t)gridDim.x * blockDim.x) {
        double2 a[RSRR_MAX_TERMS_DEV];
#pragma unroll
        for (int i = 0; i < RSRR_MAX_TERMS_DEV; ++i)
            a[i] = i < m ? A[(int64_t)i * nn2 + q] : make_double2(0.0, 0.0);
        for (int j = 0; j < nj; ++j) {
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int i = 0; i < RSRR_MAX_TERMS_DEV; ++i)
                if (i < m) acc = cfma(acc, s_cf[j * m + i], a[i]);
            T_all[(int64_t)(j0 + j) * nn2 + q] = acc;
        }
    }
}

// R(:, c) (+)= cf[c m + i] Y(:, c): one term of T(lambda_c) v_c = sum_i
// f_i(lambda_c) A_i v_c for the residuals of the dense-terms kind
__global__ void accum_term_cols_kernel(double2 *__restrict__ R, const double2 *__restrict__ Y,
                                       const double2 *__restrict__ cf, int m, int i, int n, int cnt,
                                       int first) {
    const int64_t total = (int64_t)n * cnt;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / n);
        const double2 v = cmul(cf[(size_t)c * m + i], Y[q]);
        R[q] = first ? v : cadd(R[q], v);
    }
}

// rr[c] = ||R(:, c)||_2^2 and vv[c] = ||V(:, c)||_2^2 (block per column)
__global__ void col_norms2_kernel(const double2 *__restrict__ R, const double2 *__restrict__ V, int n,
                                  double *__restrict__ rr, double *__restrict__ vv) {
    const int c = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 r = R[(int64_t)c * n + i], v = V[(int64_t)c * n + i];
        a += r.x * r.x + r.y * r.y;
        b += v.x * v.x + v.y * v.y;
    }
    __shared__ double sa[32], sb[32];
    for (int off = 16; off; off >>= 1) {
        a += shfl_down(a, off);
        b += shfl_down(b, off);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        rr[c] = ta;
        vv[c] = tb;
    }
}

// ||T(z_j)||_inf from the stored complex128 matrix: row sums of moduli
__global__ void dense_tnorm_kernel(double *__restrict__ tnorm, const double2 *__restrict__ A_all, int n) {
    const int pt = blockIdx.y;
    const double2 *A = A_all + (size_t)pt * n * n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n)
        for (int j = 0; j < n; ++j) s += cabsv(A[(int64_t)j * n + i]);
    for (int off = 16; off; off >>= 1) s = fmax(s, shfl_down(s, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(tnorm + pt, s);
}

// ---------------------------------------------------------------- LU
constexpr int DP_THREADS = 1024;
constexpr int DP_WARPS = DP_THREADS / 32;

// Panel k0 (columns k0..k0+jb-1, rows k0..n-1) of every point, one CTA per
// point, right-looking in global memory (L2): per column a block-wide argmax
// of |re|+|im| (first index on ties), the interchange inside the panel, the
// multipliers and the rank-1 update of the remaining panel columns.  Then
// the inverses of the unit lower L11 and of U11 (jb x jb) for the solve.
template <typename C, int NB>
__global__ void __launch_bounds__(DP_THREADS, 1)
dense_panel_kernel(C *__restrict__ A_all, int32_t *__restrict__ piv_all, int32_t *__restrict__ info_all,
                   C *__restrict__ dinv_all, int n, int k0) {
    using R = typename real_of<C>::type;
    const int pt = blockIdx.x;
    C *A = A_all + (size_t)pt * n * n;
    int32_t *piv = piv_all + (size_t)pt * n;
    const int jb = min(NB, n - k0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ R s_v[DP_WARPS];
    __shared__ int s_i[DP_WARPS];
    __shared__ C s_row[NB];
    __shared__ C s_blk[NB * NB];
    __shared__ C s_inv[2][NB * (NB + 1)];
    for (int cc = 0; cc < jb; ++cc) {
        const int c = k0 + cc;
        R v = (R)-1;
        int ix = 0x7fffffff;
        for (int r = c + tid; r < n; r += DP_THREADS) {
            const R a = cabs1(A[(int64_t)c * n + r]);
            if (a > v) { v = a; ix = r; }
        }
        for (int off = 16; off; off >>= 1) {
            const R ov = shfl_down(v, off);
            const int oi = shfl_down(ix, off);
            if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
        }
        if (lane == 0) { s_v[warp] = v; s_i[warp] = ix; }
        __syncthreads();
        R bv = s_v[0];
        int p = s_i[0];
        for (int w = 1; w < DP_WARPS; ++w)
            if (s_v[w] > bv || (s_v[w] == bv && s_i[w] < p)) { bv = s_v[w]; p = s_i[w]; }
        if (tid < jb && p != c) {
            const int64_t col = (int64_t)(k0 + tid) * n;
            const C t = A[col + c]; A[col + c] = A[col + p]; A[col + p] = t;
        }
        __syncthreads();
        if (tid < jb) s_row[tid] = A[(int64_t)(k0 + tid) * n + c];
        if (tid == 0) {
            piv[c] = p;
            if (!(bv > (R)0) && info_all[pt] == 0) info_all[pt] = c + 1;
        }
        __syncthreads();
        const C pv = s_row[cc];
        if (cnonzero(pv)) {
            const C inv = crecip(pv);
            for (int r = c + 1 + tid; r < n; r += DP_THREADS) {
                const C l = cmul(A[(int64_t)c * n + r], inv);
                A[(int64_t)c * n + r] = l;
                for (int c2 = cc + 1; c2 < jb; ++c2) {
                    C *a = A + (int64_t)(k0 + c2) * n + r;
                    *a = cfms(*a, l, s_row[c2]);
                }
            }
        }
        __syncthreads();
    }
    // diagonal block inverses
    for (int q = tid; q < NB * NB; q += DP_THREADS) {
        const int j = q / NB, i = q % NB;
        s_blk[q] = (i < jb && j < jb) ? A[(int64_t)(k0 + j) * n + k0 + i] : czero<C>();
    }
    __syncthreads();
    if (warp == 0 && lane < NB) {
        const int j = lane;  // column j of L11^{-1}
        for (int i = 0; i < NB; ++i) {
            C s = (i == j) ? cone<C>() : czero<C>();
            for (int t = j; t < i; ++t) s = cfms(s, s_blk[t * NB + i], s_inv[0][j * (NB + 1) + t]);
            s_inv[0][j * (NB + 1) + i] = (i < j || i >= jb || j >= jb) ? czero<C>() : s;
        }
    } else if (warp == 1 && lane < NB) {
        const int j = lane;  // column j of U11^{-1}
        for (int i = 0; i < NB; ++i) s_inv[1][j * (NB + 1) + i] = czero<C>();
        if (j < jb) {
            s_inv[1][j * (NB + 1) + j] = crecip(s_blk[j * NB + j]);
            for (int i = j - 1; i >= 0; --i) {
                C s = czero<C>();
                for (int t = i + 1; t <= j; ++t) s = cfma(s, s_blk[t * NB + i], s_inv[1][j * (NB + 1) + t]);
                s_inv[1][j * (NB + 1) + i] = cmul(csub(czero<C>(), s), crecip(s_blk[i * NB + i]));
            }
        }
    }
    __syncthreads();
    const int nblk = (n + NB - 1) / NB;
    C *dst = dinv_all + ((size_t)pt * nblk + k0 / NB) * 2 * NB * NB;
    for (int q = tid; q < 2 * NB * NB; q += DP_THREADS) {
        const int w = q / (NB * NB), e = q % (NB * NB), j = e / NB, i = e % NB;
        dst[q] = s_inv[w][j * (NB + 1) + i];
    }
}

// Trailing columns k0+jb.. in chunks of 32: the panel's interchanges (in
// order), then U12 = L11^{-1} A12 in place.
template <typename C, int NB>
__global__ void __launch_bounds__(256)
dense_laswp_trsm_kernel(C *__restrict__ A_all, const int32_t *__restrict__ piv_all,
                        const C *__restrict__ dinv_all, int n, int k0) {
    const int pt = blockIdx.y;
    C *A = A_all + (size_t)pt * n * n;
    const int32_t *piv = piv_all + (size_t)pt * n;
    const int jb = min(NB, n - k0);
    const int c0 = k0 + jb + blockIdx.x * 32;
    const int ncol = min(32, n - c0);
    if (ncol <= 0) return;
    const int nblk = (n + NB - 1) / NB;
    const C *Linv = dinv_all + ((size_t)pt * nblk + k0 / NB) * 2 * NB * NB;
    __shared__ C s_L[NB * NB];
    __shared__ C s_a[NB * 32];
    const int tid = threadIdx.x;
    for (int q = tid; q < NB * NB; q += 256) s_L[q] = Linv[q];
    if (tid < ncol) {
        const int64_t col = (int64_t)(c0 + tid) * n;
        for (int cc = 0; cc < jb; ++cc) {
            const int p = piv[k0 + cc];
            if (p != k0 + cc) {
                const C t = A[col + k0 + cc]; A[col + k0 + cc] = A[col + p]; A[col + p] = t;
            }
        }
    }
    __syncthreads();
    for (int q = tid; q < NB * 32; q += 256) {
        const int i = q % NB, c = q / NB;
        s_a[q] = (i < jb && c < ncol) ? A[(int64_t)(c0 + c) * n + k0 + i] : czero<C>();
    }
    __syncthreads();
    for (int q = tid; q < NB * 32; q += 256) {
        const int i = q % NB, c = q / NB;
        if (i < jb && c < ncol) {
            C s = czero<C>();
            for (int t = 0; t < NB; ++t) s = cfma(s, s_L[t * NB + i], s_a[c * NB + t]);
            A[(int64_t)(c0 + c) * n + k0 + i] = s;
        }
    }
}

// A22 -= L21 U12 over 64 x 64 tiles (K = jb), 256 threads with 4 x 4 outputs.
template <typename C, int NB>
__global__ void __launch_bounds__(256)
dense_gemm_update_kernel(C *__restrict__ A_all, int n, int k0) {
    const int pt = blockIdx.z;
    C *A = A_all + (size_t)pt * n * n;
    const int jb = min(NB, n - k0);
    const int r0 = k0 + jb + blockIdx.x * 64, c0 = k0 + jb + blockIdx.y * 64;
    if (r0 >= n || c0 >= n) return;
    __shared__ C s_l[NB][64 + 1];  // L21(r0+i, k0+t) at [t][i]
    __shared__ C s_u[NB][64 + 1];  // U12(k0+t, c0+j) at [t][j]
    const int tid = threadIdx.x;
    for (int q = tid; q < NB * 64; q += 256) {
        const int i = q % 64, t = q / 64;
        s_l[t][i] = (r0 + i < n && t < jb) ? A[(int64_t)(k0 + t) * n + r0 + i] : czero<C>();
        const int tt = q % NB, j = q / NB;
        s_u[tt][j] = (c0 + j < n && tt < jb) ? A[(int64_t)(c0 + j) * n + k0 + tt] : czero<C>();
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = r0 + tx + 16 * a, j = c0 + ty + 16 * b;
            acc[a][b] = (i < n && j < n) ? A[(int64_t)j * n + i] : czero<C>();
        }
#pragma unroll 4
    for (int t = 0; t < NB; ++t) {
        C lv[4], uv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) lv[a] = s_l[t][tx + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) uv[b] = s_u[t][ty + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = cfms(acc[a][b], lv[a], uv[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = r0 + tx + 16 * a, j = c0 + ty + 16 * b;
            if (i < n && j < n) A[(int64_t)j * n + i] = acc[a][b];
        }
}

// ---------------------------------------------------------------- solve
// One CTA per (point, chunk of LC right-hand sides); B (n x L per point,
// column major) is overwritten with the solution.  Forward per block: the
// block's interchanges, y = L11^{-1} b_block, rows below -= L21 y.  Backward
// per block from the end: t = y_block - U12 x_next (columns split across
// warps, partial tiles summed in shared memory), x = U11^{-1} t.
constexpr int DS_THREADS = 512;
constexpr int DS_WARPS = DS_THREADS / 32;

template <typename C, int NB, int LC>
__global__ void __launch_bounds__(DS_THREADS, 1)
dense_solve_kernel(const C *__restrict__ A_all, const int32_t *__restrict__ piv_all,
                   const C *__restrict__ dinv_all, C *__restrict__ B_all, int n, int L,
                   const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip && skip[pt]) return;
    const int col0 = blockIdx.x * LC;
    const int ncol = min(LC, L - col0);
    const C *A = A_all + (size_t)pt * n * n;
    const int32_t *piv = piv_all + (size_t)pt * n;
    const int nblk = (n + NB - 1) / NB;
    const C *dinv = dinv_all + (size_t)pt * nblk * 2 * NB * NB;
    C *B = B_all + (size_t)pt * L * n + (size_t)col0 * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ C s_D[NB * NB];
    __shared__ C s_y[NB * LC];
    __shared__ C s_part[DS_WARPS * NB * LC];
    // forward
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int jb = min(NB, n - k0);
        for (int q = tid; q < NB * NB; q += DS_THREADS) s_D[q] = dinv[(size_t)(k0 / NB) * 2 * NB * NB + q];
        if (tid < ncol) {
            for (int cc = 0; cc < jb; ++cc) {
                const int p = piv[k0 + cc];
                if (p != k0 + cc) {
                    C *a = B + (size_t)tid * n;
                    const C t = a[k0 + cc]; a[k0 + cc] = a[p]; a[p] = t;
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < NB * LC; q += DS_THREADS) {
            const int i = q % NB, c = q / NB;
            C y = czero<C>();
            if (i < jb && c < ncol) {
                for (int t = 0; t < jb; ++t) y = cfma(y, s_D[t * NB + i], B[(size_t)c * n + k0 + t]);
            }
            s_y[i * LC + c] = y;
        }
        __syncthreads();
        for (int q = tid; q < jb * LC; q += DS_THREADS) {
            const int i = q % jb, c = q / jb;
            if (c < ncol) B[(size_t)c * n + k0 + i] = s_y[i * LC + c];
        }
        for (int r = k0 + jb + tid; r < n; r += DS_THREADS) {
            C acc[LC];
#pragma unroll
            for (int c = 0; c < LC; ++c) acc[c] = c < ncol ? B[(size_t)c * n + r] : czero<C>();
            for (int t = 0; t < jb; ++t) {
                const C l = A[(int64_t)(k0 + t) * n + r];
#pragma unroll
                for (int c = 0; c < LC; ++c) acc[c] = cfms(acc[c], l, s_y[t * LC + c]);
            }
#pragma unroll
            for (int c = 0; c < LC; ++c)
                if (c < ncol) B[(size_t)c * n + r] = acc[c];
        }
        __syncthreads();
    }
    // backward
    for (int k0 = ((n - 1) / NB) * NB; k0 >= 0; k0 -= NB) {
        const int jb = min(NB, n - k0);
        const int k1 = k0 + jb;
        for (int q = tid; q < NB * NB; q += DS_THREADS)
            s_D[q] = dinv[(size_t)(k0 / NB) * 2 * NB * NB + NB * NB + q];
        C acc[LC];
#pragma unroll
        for (int c = 0; c < LC; ++c) acc[c] = czero<C>();
        if (lane < jb) {
            for (int col = k1 + warp; col < n; col += DS_WARPS) {
                const C u = A[(int64_t)col * n + k0 + lane];
#pragma unroll
                for (int c = 0; c < LC; ++c)
                    if (c < ncol) acc[c] = cfms(acc[c], u, B[(size_t)c * n + col]);
            }
        }
        if (lane < NB) {
#pragma unroll
            for (int c = 0; c < LC; ++c) s_part[(warp * NB + lane) * LC + c] = (lane < jb) ? acc[c] : czero<C>();
        }
        __syncthreads();
        for (int q = tid; q < NB * LC; q += DS_THREADS) {
            const int i = q / LC, c = q % LC;
            C t = czero<C>();
            if (i < jb && c < ncol) {
                t = B[(size_t)c * n + k0 + i];
                for (int w = 0; w < DS_WARPS; ++w) t = cadd(t, s_part[(w * NB + i) * LC + c]);
            }
            s_y[i * LC + c] = t;
        }
        __syncthreads();
        for (int q = tid; q < NB * LC; q += DS_THREADS) {
            const int i = q / LC, c = q % LC;
            if (i < jb && c < ncol) {
                C x = czero<C>();
                for (int t = 0; t < jb; ++t) x = cfma(x, s_D[t * NB + i], s_y[t * LC + c]);
                B[(size_t)c * n + k0 + i] = x;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- residual helpers
// column maxima of |R| (R n x L, may be null) and |X| for one point into rmax/xmax
__global__ void dense_colmax_kernel(const double2 *__restrict__ Rm, const double2 *__restrict__ X,
                                    int n, double *__restrict__ rmax, double *__restrict__ xmax) {
    const int l = blockIdx.x;
    double r = 0.0, x = 0.0;
    // squared moduli, one square root at the end (FP64 pipe)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (Rm) {
            const double2 v = Rm[(size_t)l * n + i];
            r = fmax(r, fma(v.x, v.x, v.y * v.y));
        }
        const double2 v = X[(size_t)l * n + i];
        x = fmax(x, fma(v.x, v.x, v.y * v.y));
    }
    for (int off = 16; off; off >>= 1) {
        r = fmax(r, shfl_down(r, off));
        x = fmax(x, shfl_down(x, off));
    }
    __shared__ double wr[32], wx[32];
    if ((threadIdx.x & 31) == 0) { wr[threadIdx.x >> 5] = r; wx[threadIdx.x >> 5] = x; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a = fmax(a, wr[q]); b = fmax(b, wx[q]); }
        rmax[l] = sqrt(a);
        xmax[l] = sqrt(b);
    }
}

// Taylor coefficients in place: A <- A o (i r)/p for p >= 1 (diagonal -> 0);
// for p == 0, A = exp(i c r)/(4 pi r) off the diagonal and diag on it.
__global__ void taylor_step_kernel(double2 *__restrict__ A, const double *__restrict__ pts,
                                   double2 c, double diag, int n, int p) {
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / n), i = (int)(q - (int64_t)j * n);
        if (i == j) {
            A[q] = make_double2(p == 0 ? diag : 0.0, 0.0);
            continue;
        }
        const double dx = pts[3 * i] - pts[3 * j], dy = pts[3 * i + 1] - pts[3 * j + 1],
                     dz = pts[3 * i + 2] - pts[3 * j + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (p == 0) {
            const double mag = exp(-c.y * r) / (kFourPi * r);
            double s, co;
            sincos(c.x * r, &s, &co);
            A[q] = make_double2(mag * co, mag * s);
        } else {
            const double2 a = A[q];
            const double f = r / p;  // multiply by i r / p
            A[q] = make_double2(-a.y * f, a.x * f);
        }
    }
}

// ||T(lam_c) v_c||^2, ||v_c||^2 and the column sums of |T(lam_c)| (for the
// 1-norm), matrix-free in FP64; thread per row i (and per column i for the sums).
__global__ void dense_eig_residual_kernel(const double2 *__restrict__ V, const double2 *__restrict__ lam,
                                          const double *__restrict__ pts, double diag, int n,
                                          double *__restrict__ rr, double *__restrict__ vv,
                                          double *__restrict__ t1) {
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double2 z = lam[c];
    double r2 = 0.0, v2 = 0.0, cs = 0.0;
    if (i < n) {
        double2 s = make_double2(0.0, 0.0);
        for (int j = 0; j < n; ++j) {
            double2 t;
            if (i == j) {
                t = make_double2(diag, 0.0);
            } else {
                const double dx = pts[3 * i] - pts[3 * j], dy = pts[3 * i + 1] - pts[3 * j + 1],
                             dz = pts[3 * i + 2] - pts[3 * j + 2];
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                const double mag = exp(-z.y * r) / (kFourPi * r);
                double sn, co;
                sincos(z.x * r, &sn, &co);
                t = make_double2(mag * co, mag * sn);
            }
            s = cfma(s, t, V[(int64_t)c * n + j]);
            cs += cabsv(t);  // |T_ij| = |T_ji|: row sum i equals column sum i
        }
        r2 = s.x * s.x + s.y * s.y;
        const double2 x = V[(int64_t)c * n + i];
        v2 = x.x * x.x + x.y * x.y;
    }
    for (int off = 16; off; off >>= 1) {
        r2 += shfl_down(r2, off);
        v2 += shfl_down(v2, off);
        cs = fmax(cs, shfl_down(cs, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(rr + c, r2);
        atomicAdd(vv + c, v2);
        atomic_max_nonneg(t1 + c, cs);
    }
}

// ================================================================ launchers
static int grid_for_d(int64_t work, int threads = 256, int cap = 152 * 16) {
    int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

cudaError_t launch_assemble_dense_c64(float2 *A, const double *pts, const double2 *zs, double diag,
                                      int n, int N, cudaStream_t s) {
    assemble_dense_c64_kernel<<<dim3(grid_for_d((int64_t)n * n, 256, 2048), N), 256, 0, s>>>(A, pts, zs,
                                                                                          diag, n);
    return cudaGetLastError();
}
cudaError_t launch_assemble_dense_c128(double2 *A, const double *pts, const double2 *zs, double diag,
                                       int n, int N, cudaStream_t s) {
    assemble_dense_c128_kernel<<<dim3(grid_for_d((int64_t)n * n, 256, 2048), N), 256, 0, s>>>(A, pts,
                                                                                           zs, diag, n);
    return cudaGetLastError();
}
cudaError_t launch_assemble_dense_terms(double2 *T, const double2 *A, const double2 *coef, int n, int N,
                                        int m, cudaStream_t s) {
    if (m < 1 || m > RSRR_MAX_TERMS_DEV) return cudaErrorInvalidValue;
    const int64_t nn2 = (int64_t)n * n;
    const int chunk = std::max(1, 2048 / m);  // coefficients of a chunk: <= 32 KB of shared memory
    for (int j0 = 0; j0 < N; j0 += chunk) {
        const int nj = std::min(chunk, N - j0);
        assemble_dense_terms_kernel<<<grid_for_d(nn2, 256, 152 * 8), 256, sizeof(double2) * nj * m, s>>>(
            T, A, coef, nn2, j0, nj, m);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t launch_accum_term_cols(double2 *R, const double2 *Y, const double2 *cf, int m, int i, int n,
                                   int cnt, bool first, cudaStream_t s) {
    accum_term_cols_kernel<<<grid_for_d((int64_t)n * cnt), 256, 0, s>>>(R, Y, cf, m, i, n, cnt, first ? 1 : 0);
    return cudaGetLastError();
}
cudaError_t launch_col_norms2(const double2 *R, const double2 *V, int n, int cnt, double *rr, double *vv,
                              cudaStream_t s) {
    if (cnt < 1) return cudaSuccess;
    col_norms2_kernel<<<cnt, 256, 0, s>>>(R, V, n, rr, vv);
    return cudaGetLastError();
}
cudaError_t launch_dense_tnorm(double *tnorm, const double2 *A, int n, int N, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tnorm, 0, sizeof(double) * N, s);
    if (e != cudaSuccess) return e;
    dense_tnorm_kernel<<<dim3((n + 255) / 256, N), 256, 0, s>>>(tnorm, A, n);
    return cudaGetLastError();
}

cudaError_t launch_dense_tc_update(float2 *A, int n, int k0, int jb, int N, unsigned int *status,
                                   cudaStream_t s);

// the trailing update A22 -= L21 U12 of one panel: FP32 / FP64 FMAs, or, for
// complex64 with tc, the 3xTF32 tensor-core kernel of dense_tc.cu
template <typename C, int NB>
static cudaError_t dense_update(C *A, int n, int k0, int N, unsigned int *status, bool tc, cudaStream_t s) {
    const int jb = std::min(NB, n - k0), rest = n - k0 - jb;
    if constexpr (std::is_same<C, float2>::value)
        if (tc) return launch_dense_tc_update(A, n, k0, jb, N, status, s);
    dense_gemm_update_kernel<C, NB><<<dim3((rest + 63) / 64, (rest + 63) / 64, N), 256, 0, s>>>(A, n, k0);
    return cudaGetLastError();
}

template <typename C, int NB>
static cudaError_t dense_lu_t(C *A, int32_t *piv, int32_t *info, C *dinv, int n, int N, cudaStream_t s,
                              int64_t *launches, unsigned int *status, bool tc) {
    cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int32_t) * N, s);
    if (e != cudaSuccess) return e;
    for (int k0 = 0; k0 < n; k0 += NB) {
        const int jb = std::min(NB, n - k0);
        dense_panel_kernel<C, NB><<<N, DP_THREADS, 0, s>>>(A, piv, info, dinv, n, k0);
        const int rest = n - k0 - jb;
        if (rest > 0) {
            dense_laswp_trsm_kernel<C, NB><<<dim3((rest + 31) / 32, N), 256, 0, s>>>(A, piv, dinv, n, k0);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = dense_update<C, NB>(A, n, k0, N, status, tc, s)) != cudaSuccess) return e;
            *launches += 2;
        }
        *launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_dense_lu_c64(float2 *A, int32_t *piv, int32_t *info, float2 *dinv, int n, int N,
                                cudaStream_t s, int64_t *launches, unsigned int *status, bool tc) {
    return dense_lu_t<float2, NB_C64>(A, piv, info, dinv, n, N, s, launches, status, tc);
}
cudaError_t launch_dense_lu_c128(double2 *A, int32_t *piv, int32_t *info, double2 *dinv, int n, int N,
                                 cudaStream_t s, int64_t *launches) {
    return dense_lu_t<double2, NB_C128>(A, piv, info, dinv, n, N, s, launches, nullptr, false);
}

cudaError_t launch_dense_solve_c64(const float2 *A, const int32_t *piv, const float2 *dinv, float2 *B,
                                   int n, int N, int L, const int32_t *skip, cudaStream_t s) {
    dense_solve_kernel<float2, NB_C64, 8><<<dim3((L + 7) / 8, N), DS_THREADS, 0, s>>>(A, piv, dinv, B, n,
                                                                                      L, skip);
    return cudaGetLastError();
}
cudaError_t launch_dense_solve_c128(const double2 *A, const int32_t *piv, const double2 *dinv,
                                    double2 *B, int n, int N, int L, const int32_t *skip,
                                    cudaStream_t s) {
    dense_solve_kernel<double2, NB_C128, 8><<<dim3((L + 7) / 8, N), DS_THREADS, 0, s>>>(A, piv, dinv, B, n,
                                                                                       L, skip);
    return cudaGetLastError();
}

cudaError_t launch_dense_colmax(const double2 *R, const double2 *X, int n, int L, double *rmax,
                                double *xmax, cudaStream_t s) {
    dense_colmax_kernel<<<L, 256, 0, s>>>(R, X, n, rmax, xmax);
    return cudaGetLastError();
}

cudaError_t launch_taylor_step(double2 *A, const double *pts, double2 c, double diag, int n, int p,
                               cudaStream_t s) {
    taylor_step_kernel<<<grid_for_d((int64_t)n * n, 256, 4096), 256, 0, s>>>(A, pts, c, diag, n, p);
    return cudaGetLastError();
}

cudaError_t launch_dense_eig_residual(const double2 *V, const double2 *lam, const double *pts,
                                      double diag, int n, int cnt, double *rr, double *vv, double *t1,
                                      cudaStream_t s) {
    dense_eig_residual_kernel<<<dim3((n + 127) / 128, cnt), 128, 0, s>>>(V, lam, pts, diag, n, rr, vv, t1);
    return cudaGetLastError();
}

}  // namespace rsrr
