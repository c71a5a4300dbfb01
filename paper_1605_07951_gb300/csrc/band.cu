// Resolvent sampling on banded T(z_j) (RSRR step 2, Section 3.3):
//   assembly of T(z_j) = sum_i f_i(z_j) A_i into band LU storage,
//   batched banded LU with partial pivoting (one CTA per sampling point),
//   blocked triangular solves for the L probe columns,
//   FP64 residual r = U - T(z_j) X with per-column backward errors, and the
//   refinement updates of the mixed-precision path.
//
// Band storage of one point (column major, leading dimension ldab):
//   A(i, c) lives at ab[c * ldab + KV + i - c], KV = kl + ku, for
//   c - KV <= i <= c + kl + NB - 1,  ldab = KV + kl + NB.
// Rows above the original band hold the fill of partial pivoting (upper
// bandwidth grows to kl + ku); the NB - 1 rows below the lower band hold the
// multipliers that later row interchanges inside the same NB-column block
// move down (pivoting is applied dense-style within a block).  The solve
// walks the same blocks, so the factor and the solve agree on NB.
#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

RSRR_DEV void store_c(float2 *p, double2 v) { *p = to_c64(v); }
RSRR_DEV void store_c(double2 *p, double2 v) { *p = v; }

// --------------------------------------------------------------------------
// Assembly: one thread per stored band entry (column c, band row t) of one
// point.  The value is sum_q coef[pt][q] * vals[q][e] for the pattern entry
// e = (i, c), found by binary search in column c of a CSC copy of the
// pattern; every other stored entry (fill rows, zeros) is written as zero.
// --------------------------------------------------------------------------
template <typename C>
__global__ void assemble_band_kernel(C *__restrict__ ab_all, const double2 *__restrict__ coef,
                                     const int32_t *__restrict__ csc_ptr,
                                     const int32_t *__restrict__ csc_row,
                                     const int32_t *__restrict__ csc_perm,
                                     const double *__restrict__ vals, int64_t nnz, int m, int n,
                                     int kl, int ku, int ldab) {
    const int pt = blockIdx.y;
    const int64_t total = (int64_t)ldab * n;
    const int KV = kl + ku;
    C *ab = ab_all + (size_t)pt * total;
    __shared__ double2 s_coef[RSRR_MAX_TERMS_DEV];
    if (threadIdx.x < m) s_coef[threadIdx.x] = coef[pt * m + threadIdx.x];
    __syncthreads();
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / ldab);
        const int t = (int)(idx - (int64_t)c * ldab);
        const int i = c + t - KV;
        double2 v = make_double2(0.0, 0.0);
        if (i >= 0 && i < n && i - c <= kl && c - i <= ku) {
            int lo = csc_ptr[c], hi = csc_ptr[c + 1];
            const int end = hi;
            while (lo < hi) {  // first entry of column c with row >= i
                const int mid = (lo + hi) >> 1;
                if (csc_row[mid] < i) lo = mid + 1; else hi = mid;
            }
            if (lo < end && csc_row[lo] == i) {
                const int64_t e = csc_perm[lo];
                for (int q = 0; q < m; ++q) {
                    const double a = vals[(int64_t)q * nnz + e];
                    v.x = fma(s_coef[q].x, a, v.x);
                    v.y = fma(s_coef[q].y, a, v.y);
                }
            }
        }
        store_c(ab + idx, v);
    }
}

// ||T(z_j)||_inf = max_i sum_c |t_ic| (modulus), from the CSR pattern in FP64.
__global__ void tnorm_kernel(double *__restrict__ tnorm, const double2 *__restrict__ coef,
                             const int32_t *__restrict__ row_ptr, const double *__restrict__ vals,
                             int64_t nnz, int m, int n) {
    const int pt = blockIdx.y;
    __shared__ double2 s_coef[RSRR_MAX_TERMS_DEV];
    if (threadIdx.x < m) s_coef[threadIdx.x] = coef[pt * m + threadIdx.x];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            double2 v = make_double2(0.0, 0.0);
            for (int q = 0; q < m; ++q) {
                const double a = vals[(int64_t)q * nnz + e];
                v.x = fma(s_coef[q].x, a, v.x);
                v.y = fma(s_coef[q].y, a, v.y);
            }
            s += hypot(v.x, v.y);
        }
    }
    for (int off = 16; off; off >>= 1) s = fmax(s, shfl_down(s, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(tnorm + pt, s);
}

// --------------------------------------------------------------------------
// Blocked solve with the factors of band_lu_kernel, one CTA per (point,
// chunk of LC right-hand sides), B overwritten with the solution.
// Forward: per NB block, the block's interchanges then unit-lower
// elimination over the block rows (rows j0..j0+pr-1 live in a shared-memory
// window).  Backward: column-oriented back substitution with the upper band
// (bandwidth kl+ku), rows [c-KV, c] in a shared-memory window.
// Points with skip[pt] != 0 are left untouched.
// --------------------------------------------------------------------------
constexpr int SV_THREADS = 512;

template <typename C, int NB, int LC>
__global__ void __launch_bounds__(SV_THREADS, 1)
band_solve_kernel(const C *__restrict__ ab_all, const int32_t *__restrict__ piv_all,
                  C *__restrict__ B_all, int n, int kl, int ku, int ldab, int L,
                  const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip && skip[pt]) return;
    const int col0 = blockIdx.x * LC;
    const int ncol = min(LC, L - col0);
    const C *ab = ab_all + (size_t)pt * ldab * n;
    const int32_t *piv = piv_all + (size_t)pt * n;
    C *B = B_all + (size_t)pt * L * n + (size_t)col0 * n;
    const int KV = kl + ku;
    const int tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *W = reinterpret_cast<C *>(smem_raw);  // [WR][LC] circular window, row-major by slot
    const int WF = kl + NB;                  // forward window rows
    const int WB = KV + NB;                  // backward window rows
    const int WR = WF > WB ? WF : WB;

    // ---------------- forward
    int loaded = 0;  // rows [.., loaded) are in the window
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = min(NB, n - j0);
        const int pr = min(n - j0, jb + kl);
        const int need = j0 + pr;
        for (int o = tid; o < (need - loaded) * LC; o += SV_THREADS) {
            const int i = loaded + o / LC, col = o % LC;
            W[(i % WR) * LC + col] = col < ncol ? B[(size_t)col * n + i] : czero<C>();
        }
        loaded = max(loaded, need);
        __syncthreads();
        if (tid < ncol) {
            for (int cc = 0; cc < jb; ++cc) {
                const int p = piv[j0 + cc];
                if (p != j0 + cc) {
                    C *a = W + ((j0 + cc) % WR) * LC + tid;
                    C *b = W + (p % WR) * LC + tid;
                    const C t = *a; *a = *b; *b = t;
                }
            }
        }
        __syncthreads();
        for (int cc = 0; cc < jb; ++cc) {
            const int c = j0 + cc;
            const int nrow = pr - cc - 1;  // rows c+1 .. j0+pr-1
            for (int o = tid; o < nrow * LC; o += SV_THREADS) {
                const int r = o % nrow, col = o / nrow;
                const int i = c + 1 + r;
                if (col < ncol) {
                    const C l = ab[(size_t)c * ldab + KV + (i - c)];
                    const C y = W[(c % WR) * LC + col];
                    C *w = W + (i % WR) * LC + col;
                    *w = cfms(*w, l, y);
                }
            }
            __syncthreads();
        }
        for (int o = tid; o < jb * LC; o += SV_THREADS) {
            const int i = j0 + o / LC, col = o % LC;
            if (col < ncol) B[(size_t)col * n + i] = W[(i % WR) * LC + col];
        }
        __syncthreads();
    }
    // ---------------- backward
    int low = n;  // rows [low, ..) are in the window
    for (int j1 = n; j1 > 0; j1 -= NB) {
        const int j0 = max(0, j1 - NB);
        const int need = max(0, j0 - KV);
        for (int o = tid; o < (low - need) * LC; o += SV_THREADS) {
            const int i = need + o / LC, col = o % LC;
            W[(i % WR) * LC + col] = col < ncol ? B[(size_t)col * n + i] : czero<C>();
        }
        low = min(low, need);
        __syncthreads();
        for (int c = j1 - 1; c >= j0; --c) {
            const C inv = crecip(ab[(size_t)c * ldab + KV]);
            const int i0 = max(0, c - KV);
            const int nrow = c - i0;
            // x_c = w_c / u_cc is formed by every thread from the window
            for (int o = tid; o < nrow * LC; o += SV_THREADS) {
                const int r = o % nrow, col = o / nrow;
                const int i = i0 + r;
                if (col < ncol) {
                    const C x = cmul(W[(c % WR) * LC + col], inv);
                    const C u = ab[(size_t)c * ldab + KV + (i - c)];
                    C *w = W + (i % WR) * LC + col;
                    *w = cfms(*w, u, x);
                }
            }
            __syncthreads();
            if (tid < ncol) {
                C *w = W + (c % WR) * LC + tid;
                *w = cmul(*w, inv);
            }
            __syncthreads();
        }
        for (int o = tid; o < (j1 - j0) * LC; o += SV_THREADS) {
            const int i = j0 + o / LC, col = o % LC;
            if (col < ncol) B[(size_t)col * n + i] = W[(i % WR) * LC + col];
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// FP64 residual R = U - T(z_j) X for LCH columns per thread (CSR, on the fly
// coefficients), with column maxima of |R| and |X| for the backward errors.
// Points with skip[pt] != 0 are skipped.  R may be null (statistics only).
// --------------------------------------------------------------------------
constexpr int RES_LCH = 8;

__global__ void residual_kernel(double2 *__restrict__ R, const double2 *__restrict__ X,
                                const double2 *__restrict__ U, const double2 *__restrict__ coef,
                                const int32_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col_idx,
                                const double *__restrict__ vals, int64_t nnz, int m, int n, int L,
                                double *__restrict__ rmax, double *__restrict__ xmax,
                                const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip && skip[pt]) return;
    __shared__ double2 s_coef[RSRR_MAX_TERMS_DEV];
    if (threadIdx.x < m) s_coef[threadIdx.x] = coef[pt * m + threadIdx.x];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int l0 = blockIdx.z * RES_LCH;
    const double2 *Xp = X + (size_t)pt * L * n;
    double2 acc[RES_LCH];
    double xm[RES_LCH];
#pragma unroll
    for (int l = 0; l < RES_LCH; ++l) {
        acc[l] = make_double2(0.0, 0.0);
        xm[l] = 0.0;
        if (i < n && l0 + l < L) {
            acc[l] = U[(size_t)(l0 + l) * n + i];
            xm[l] = cabsv(Xp[(size_t)(l0 + l) * n + i]);
        }
    }
    if (i < n) {
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            double2 a = make_double2(0.0, 0.0);
            for (int q = 0; q < m; ++q) {
                const double v = vals[(int64_t)q * nnz + e];
                a.x = fma(s_coef[q].x, v, a.x);
                a.y = fma(s_coef[q].y, v, a.y);
            }
            const int c = col_idx[e];
#pragma unroll
            for (int l = 0; l < RES_LCH; ++l)
                if (l0 + l < L) acc[l] = cfms(acc[l], a, Xp[(size_t)(l0 + l) * n + c]);
        }
    }
#pragma unroll
    for (int l = 0; l < RES_LCH; ++l) {
        if (R && i < n && l0 + l < L) R[(size_t)pt * L * n + (size_t)(l0 + l) * n + i] = acc[l];
        double rv = cabsv(acc[l]), xv = xm[l];
        for (int off = 16; off; off >>= 1) {
            rv = fmax(rv, shfl_down(rv, off));
            xv = fmax(xv, shfl_down(xv, off));
        }
        if ((threadIdx.x & 31) == 0 && l0 + l < L) {
            atomic_max_nonneg(rmax + pt * L + l0 + l, rv);
            atomic_max_nonneg(xmax + pt * L + l0 + l, xv);
        }
    }
}

// eta per column; done[pt] = all L columns of the point at or below eta_tol.
// *sweeps is set to 1 if some point is not done.  Skipped points keep their
// previous eta and done flag.
__global__ void eta_kernel(double *__restrict__ eta, int32_t *__restrict__ done,
                           const double *__restrict__ rmax, const double *__restrict__ xmax,
                           const double *__restrict__ umax, const double *__restrict__ tnorm,
                           int N, int L, double tol, int32_t *__restrict__ sweeps,
                           const int32_t *__restrict__ skip) {
    const int pt = blockIdx.x;
    if (skip && skip[pt]) return;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const double den = tnorm[pt] * xmax[pt * L + l] + umax[l];
        const double e = den > 0.0 ? rmax[pt * L + l] / den : 0.0;
        eta[pt * L + l] = e;
        if (!(e <= tol)) atomicOr(&s_bad, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        done[pt] = s_bad ? 0 : 1;
        if (s_bad && sweeps) atomicOr(sweeps, 1);
    }
}

// column maxima of |U| (once per probe)
__global__ void colmax_kernel(double *__restrict__ out, const double2 *__restrict__ U, int n, int L) {
    const int l = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, cabsv(U[(size_t)l * n + i]));
    for (int off = 16; off; off >>= 1) s = fmax(s, shfl_down(s, off));
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, w[q]);
        out[l] = r;
    }
}

// D[pt] = (C) U for every point (initial right-hand sides)
template <typename C>
__global__ void broadcast_probe_kernel(C *__restrict__ D, const double2 *__restrict__ U,
                                       int64_t nL, int N) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nL * N;
         q += (int64_t)gridDim.x * blockDim.x)
        store_c(D + q, U[q % nL]);
}

// X = (c128) D for all points
__global__ void widen_kernel(double2 *__restrict__ X, const float2 *__restrict__ D, int64_t total) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        X[q] = to_c128(D[q]);
}

// D = (c64) R for points still refining
__global__ void narrow_kernel(float2 *__restrict__ D, const double2 *__restrict__ R, int64_t per_pt,
                              int N, const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip[pt]) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < per_pt;
         q += (int64_t)gridDim.x * blockDim.x)
        D[pt * per_pt + q] = to_c64(R[pt * per_pt + q]);
}

// X += D for points still refining
__global__ void update_kernel(double2 *__restrict__ X, const float2 *__restrict__ D, int64_t per_pt,
                              int N, const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip[pt]) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < per_pt;
         q += (int64_t)gridDim.x * blockDim.x) {
        const float2 d = D[pt * per_pt + q];
        double2 x = X[pt * per_pt + q];
        x.x += (double)d.x;
        x.y += (double)d.y;
        X[pt * per_pt + q] = x;
    }
}

// ==========================================================================
// launchers
// ==========================================================================
static int grid_for(int64_t work, int threads, int cap = 152 * 16) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

template <typename C>
cudaError_t launch_assemble(C *ab, const BandGeom &g, const DevProblem &p, cudaStream_t s) {
    const int64_t total = (int64_t)g.ldab * p.n;
    dim3 grid(grid_for(total, 256, 4096), p.N);
    assemble_band_kernel<C><<<grid, 256, 0, s>>>(ab, p.coef, p.csc_ptr, p.csc_row, p.csc_perm,
                                                 p.vals, p.nnz, p.m, (int)p.n, g.kl, g.ku, g.ldab);
    return cudaGetLastError();
}

cudaError_t launch_tnorm(double *tnorm, const DevProblem &p, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tnorm, 0, sizeof(double) * p.N, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.n + 255) / 256), p.N);
    tnorm_kernel<<<grid, 256, 0, s>>>(tnorm, p.coef, p.row_ptr, p.vals, p.nnz, p.m, (int)p.n);
    return cudaGetLastError();
}

template <typename C, int NB, int LC>
static cudaError_t solve_dispatch(const C *ab, const int32_t *piv, C *B, const BandGeom &g, int N,
                                  int n, int L, const int32_t *skip, cudaStream_t s) {
    const int WR = max(g.kl + NB, g.kl + g.ku + NB);
    const size_t smem = sizeof(C) * (size_t)WR * LC;
    cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<C, NB, LC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((L + LC - 1) / LC, N);
    band_solve_kernel<C, NB, LC><<<grid, SV_THREADS, smem, s>>>(ab, piv, B, n, g.kl, g.ku, g.ldab,
                                                                 L, skip);
    return cudaGetLastError();
}

cudaError_t launch_band_solve_c64(const float2 *ab, const int32_t *piv, float2 *B, const BandGeom &g,
                                  int N, int n, int L, const int32_t *skip, cudaStream_t s) {
    return solve_dispatch<float2, NB_C64, 16>(ab, piv, B, g, N, n, L, skip, s);
}
cudaError_t launch_band_solve_c128(const double2 *ab, const int32_t *piv, double2 *B,
                                   const BandGeom &g, int N, int n, int L, const int32_t *skip,
                                   cudaStream_t s) {
    return solve_dispatch<double2, NB_C128, 8>(ab, piv, B, g, N, n, L, skip, s);
}

cudaError_t launch_residual(double2 *R, const double2 *X, const DevProblem &p, double *rmax,
                            double *xmax, const int32_t *skip, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(rmax, 0, sizeof(double) * p.N * p.L, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(xmax, 0, sizeof(double) * p.N * p.L, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.n + 127) / 128), p.N, (p.L + RES_LCH - 1) / RES_LCH);
    residual_kernel<<<grid, 128, 0, s>>>(R, X, p.U, p.coef, p.row_ptr, p.col_idx, p.vals, p.nnz,
                                         p.m, (int)p.n, p.L, rmax, xmax, skip);
    return cudaGetLastError();
}

cudaError_t launch_eta(double *eta, int32_t *done, const double *rmax, const double *xmax,
                       const double *umax, const double *tnorm, int N, int L, double tol,
                       int32_t *sweeps, const int32_t *skip, cudaStream_t s) {
    eta_kernel<<<N, 128, 0, s>>>(eta, done, rmax, xmax, umax, tnorm, N, L, tol, sweeps, skip);
    return cudaGetLastError();
}

cudaError_t launch_colmax(double *out, const double2 *U, int n, int L, cudaStream_t s) {
    colmax_kernel<<<L, 256, 0, s>>>(out, U, n, L);
    return cudaGetLastError();
}

cudaError_t launch_broadcast_probe_c64(float2 *D, const double2 *U, int64_t nL, int N,
                                       cudaStream_t s) {
    broadcast_probe_kernel<float2><<<grid_for(nL * N, 256), 256, 0, s>>>(D, U, nL, N);
    return cudaGetLastError();
}
cudaError_t launch_broadcast_probe_c128(double2 *D, const double2 *U, int64_t nL, int N,
                                        cudaStream_t s) {
    broadcast_probe_kernel<double2><<<grid_for(nL * N, 256), 256, 0, s>>>(D, U, nL, N);
    return cudaGetLastError();
}
cudaError_t launch_widen(double2 *X, const float2 *D, int64_t total, cudaStream_t s) {
    widen_kernel<<<grid_for(total, 256), 256, 0, s>>>(X, D, total);
    return cudaGetLastError();
}
cudaError_t launch_narrow(float2 *D, const double2 *R, int64_t per_pt, int N, const int32_t *skip,
                          cudaStream_t s) {
    dim3 grid(grid_for(per_pt, 256, 64), N);
    narrow_kernel<<<grid, 256, 0, s>>>(D, R, per_pt, N, skip);
    return cudaGetLastError();
}
cudaError_t launch_update(double2 *X, const float2 *D, int64_t per_pt, int N, const int32_t *skip,
                          cudaStream_t s) {
    dim3 grid(grid_for(per_pt, 256, 64), N);
    update_kernel<<<grid, 256, 0, s>>>(X, D, per_pt, N, skip);
    return cudaGetLastError();
}

template cudaError_t launch_assemble<float2>(float2 *, const BandGeom &, const DevProblem &,
                                             cudaStream_t);
template cudaError_t launch_assemble<double2>(double2 *, const BandGeom &, const DevProblem &,
                                              cudaStream_t);

}  // namespace rsrr
