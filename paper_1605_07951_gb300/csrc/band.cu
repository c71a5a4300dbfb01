// Resolvent sampling on banded T(z_j) (RSRR step 2, Section 4.3):
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
#include <algorithm>

#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

RSRR_DEV void store_c(float2 *p, double2 v) { *p = to_c64(v); }
RSRR_DEV void store_c(double2 *p, double2 v) { *p = v; }
// real storage (real NEP at real points: the imaginary parts are zero)
RSRR_DEV void store_c(float *p, double2 v) { *p = (float)v.x; }
RSRR_DEV void store_c(double *p, double2 v) { *p = v.x; }

// --------------------------------------------------------------------------
// Assembly: one warp per column c of one point.  The warp first writes the
// whole stored column (ldab entries, fill rows and zeros) as zero with
// coalesced stores, then, after a warp barrier that orders the two passes,
// writes each pattern entry e = (i, c) of the column (a CSC copy of the
// pattern) at band row KV + i - c as sum_q coef[pt][q] * vals[q][e].  The
// second pass touches lines the first just wrote, so DRAM sees one write
// stream of the band storage.
// --------------------------------------------------------------------------
template <typename C>
__global__ void assemble_band_kernel(C *__restrict__ ab_all, const double2 *__restrict__ coef,
                                     const int32_t *__restrict__ csc_ptr,
                                     const int32_t *__restrict__ csc_row,
                                     const int32_t *__restrict__ csc_perm,
                                     const double *__restrict__ vals, int64_t nnz, int m, int n,
                                     int kl, int ku, int ldab) {
    const int pt = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int KV = kl + ku;
    C *ab = ab_all + (size_t)pt * ldab * n;
    __shared__ double2 s_coef[RSRR_MAX_TERMS_DEV];
    if (threadIdx.x < m) s_coef[threadIdx.x] = coef[pt * m + threadIdx.x];
    __syncthreads();
    for (int c = blockIdx.x * warps + (threadIdx.x >> 5); c < n; c += gridDim.x * warps) {
        C *col = ab + (size_t)c * ldab;
        for (int t = lane; t < ldab; t += 32) store_c(col + t, make_double2(0.0, 0.0));
        __syncwarp();
        for (int k = csc_ptr[c] + lane; k < csc_ptr[c + 1]; k += 32) {
            const int i = csc_row[k];
            if (i - c > kl || c - i > ku) continue;
            const int64_t e = csc_perm[k];
            double2 v = make_double2(0.0, 0.0);
            for (int q = 0; q < m; ++q) {
                const double a = vals[(int64_t)q * nnz + e];
                v.x = fma(s_coef[q].x, a, v.x);
                v.y = fma(s_coef[q].y, a, v.y);
            }
            store_c(col + (KV + i - c), v);
        }
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
// chunk of LC right-hand sides); B is overwritten with the solution.
// Rows live in a circular shared-memory window W[slot][LC] (row major, so
// a thread reads the LC values of one row as broadcast vector loads).
// Forward, per NB block (rows j0..j0+pr-1): gather the block's row
// permutation into G, y = L11^{-1} G_top, then G_below - L21 y with L21
// staged through shared memory (lane = row, each warp a row group and half
// of the columns, register accumulators).
// Backward, per block from the end: t = y_block - U12 x_next with U12 staged
// in column chunks; the K dimension (columns of U12) is split across warps,
// each warp accumulates a full NB x LC tile in registers (lane = row), and the
// partial tiles are summed through shared memory; then x = U11^{-1} t.
// The diagonal-block inverses come from the factorisation.  Points with
// skip[pt] != 0 are left untouched.
// --------------------------------------------------------------------------
constexpr int SV_THREADS = 512;
constexpr int SV_WARPS = SV_THREADS / 32;
constexpr int SV_FCH = 256;  // forward: rows of L21 per staged chunk
constexpr int SV_BCH = 128;  // backward: columns of U12 per staged chunk

template <typename C, int NB, int LC>
__global__ void __launch_bounds__(SV_THREADS, 1)
band_solve_kernel(const C *__restrict__ ab_all, const int32_t *__restrict__ piv_all,
                  const C *__restrict__ dinv_all, C *__restrict__ B_all, int n, int kl, int ku,
                  int ldab, int L, const int32_t *__restrict__ skip) {
    static_assert(NB <= 32, "one lane per block row");
    constexpr int HC = LC / 2;  // columns per warp in the forward update
    const int pt = blockIdx.y;
    if (skip && skip[pt]) return;
    const int col0 = blockIdx.x * LC;
    const int ncol = min(LC, L - col0);
    const int nblk = (n + NB - 1) / NB;
    const C *ab = ab_all + (size_t)pt * ldab * n;
    const int32_t *piv = piv_all + (size_t)pt * n;
    const C *dinv = dinv_all + (size_t)pt * nblk * 2 * NB * NB;
    C *B = B_all + (size_t)pt * L * n + (size_t)col0 * n;
    const int KV = kl + ku;
    const int WR = KV + NB;  // >= kl + NB
    const int PRM = NB + kl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *W = reinterpret_cast<C *>(smem_raw);  // [WR][LC]
    C *G = W + (size_t)WR * LC;              // forward [PRM][LC]; backward partials [SV_WARPS][NB][LC]
    const int GSZ = max(PRM * LC, SV_WARPS * NB * LC);
    C *St = G + GSZ;                         // [NB][SV_FCH] fwd or [SV_BCH][NB] bwd
    C *D = St + NB * SV_FCH;                 // [NB][NB]
    C *Yb = D + NB * NB;                     // [NB][LC]
    int *perm = reinterpret_cast<int *>(Yb + NB * LC);  // [PRM]

    // ---------------- forward: y = L^{-1} P b, block by block
    int loaded = 0;
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = min(NB, n - j0);
        const int pr = min(n - j0, jb + kl);
        const int need = j0 + pr;
        const int nl = need - loaded;
        for (int o = tid; o < nl * LC; o += SV_THREADS) {
            const int r = o % nl, col = o / nl;
            const int i = loaded + r;
            W[(i % WR) * LC + col] = col < ncol ? B[(size_t)col * n + i] : czero<C>();
        }
        loaded = max(loaded, need);
        for (int r = tid; r < pr; r += SV_THREADS) perm[r] = r;
        for (int q = tid; q < NB * NB; q += SV_THREADS) D[q] = dinv[(size_t)(j0 / NB) * 2 * NB * NB + q];
        __syncthreads();
        if (tid == 0) {
            for (int cc = 0; cc < jb; ++cc) {
                const int p = piv[j0 + cc] - j0;
                const int t = perm[cc]; perm[cc] = perm[p]; perm[p] = t;
            }
        }
        __syncthreads();
        for (int o = tid; o < pr * LC; o += SV_THREADS) {
            const int r = o / LC, col = o % LC;
            G[r * LC + col] = W[((j0 + perm[r]) % WR) * LC + col];
        }
        __syncthreads();
        // y = L11^{-1} G_top  (thread = (row, column))
        for (int o = tid; o < NB * LC; o += SV_THREADS) {
            const int r = o / LC, col = o % LC;
            C y = czero<C>();
            if (r < jb) {
                for (int t = 0; t < jb; ++t) y = cfma(y, D[t * NB + r], G[t * LC + col]);
                W[((j0 + r) % WR) * LC + col] = y;
            }
            Yb[r * LC + col] = y;
        }
        __syncthreads();
        // rows below: G_below - L21 y
        for (int r0 = jb; r0 < pr; r0 += SV_FCH) {
            const int ch = min(SV_FCH, pr - r0);
            for (int o = tid; o < ch * NB; o += SV_THREADS) {
                const int rr = o % ch, t = o / ch;
                C v = czero<C>();
                if (t < jb) v = ab[(size_t)(j0 + t) * ldab + KV + (r0 + rr - t)];
                St[t * SV_FCH + rr] = v;
            }
            __syncthreads();
            // warp w: rows (w % (SV_WARPS/2))*32 + lane (+ multiples), columns half (w / 8)
            const int hw = warp / (SV_WARPS / 2), rg = warp % (SV_WARPS / 2);
            for (int rr = rg * 32 + lane; rr < ch; rr += (SV_WARPS / 2) * 32) {
                C acc[HC];
#pragma unroll
                for (int c = 0; c < HC; ++c) acc[c] = G[(r0 + rr) * LC + hw * HC + c];
#pragma unroll 4
                for (int t = 0; t < NB; ++t) {
                    const C l = St[t * SV_FCH + rr];
#pragma unroll
                    for (int c = 0; c < HC; ++c) acc[c] = cfms(acc[c], l, Yb[t * LC + hw * HC + c]);
                }
#pragma unroll
                for (int c = 0; c < HC; ++c) W[((j0 + r0 + rr) % WR) * LC + hw * HC + c] = acc[c];
            }
            __syncthreads();
        }
        for (int o = tid; o < jb * LC; o += SV_THREADS) {
            const int r = o % jb, col = o / jb;
            if (col < ncol) B[(size_t)col * n + j0 + r] = W[((j0 + r) % WR) * LC + col];
        }
        __syncthreads();
    }
    // ---------------- backward: x = U^{-1} y, blocks from the end
    const int nlast = (nblk - 1) * NB;
    for (int j0 = nlast; j0 >= 0; j0 -= NB) {
        const int jb = min(NB, n - j0);
        const int j1 = j0 + jb;
        for (int o = tid; o < jb * LC; o += SV_THREADS) {
            const int r = o % jb, col = o / jb;
            W[((j0 + r) % WR) * LC + col] = col < ncol ? B[(size_t)col * n + j0 + r] : czero<C>();
        }
        for (int q = tid; q < NB * NB; q += SV_THREADS)
            D[q] = dinv[(size_t)(j0 / NB) * 2 * NB * NB + NB * NB + q];
        C acc[LC];
#pragma unroll
        for (int c = 0; c < LC; ++c) acc[c] = czero<C>();
        const int cend = min(n, j1 + KV);
        for (int c0 = j1; c0 < cend; c0 += SV_BCH) {
            const int ch = min(SV_BCH, cend - c0);
            __syncthreads();
            for (int o = tid; o < ch * NB; o += SV_THREADS) {
                const int r = o % NB, cc = o / NB;
                C v = czero<C>();
                const int d = j0 + r - (c0 + cc);
                if (r < jb && d >= -KV) v = ab[(size_t)(c0 + cc) * ldab + KV + d];
                St[cc * NB + r] = v;
            }
            __syncthreads();
            if (lane < NB) {
                for (int cc = warp; cc < ch; cc += SV_WARPS) {
                    const C u = St[cc * NB + lane];
                    const C *xr = W + ((c0 + cc) % WR) * LC;
#pragma unroll
                    for (int c = 0; c < LC; ++c) acc[c] = cfms(acc[c], u, xr[c]);
                }
            }
        }
        __syncthreads();
        if (lane < NB) {
#pragma unroll
            for (int c = 0; c < LC; ++c) G[(warp * NB + lane) * LC + c] = acc[c];
        }
        __syncthreads();
        for (int o = tid; o < NB * LC; o += SV_THREADS) {
            const int r = o / LC, col = o % LC;
            C t = czero<C>();
            if (r < jb) {
                t = W[((j0 + r) % WR) * LC + col];
                for (int w = 0; w < SV_WARPS; ++w) t = cadd(t, G[(w * NB + r) * LC + col]);
            }
            Yb[r * LC + col] = t;
        }
        __syncthreads();
        for (int o = tid; o < NB * LC; o += SV_THREADS) {
            const int r = o / LC, col = o % LC;
            if (r < jb) {
                C x = czero<C>();
#pragma unroll 8
                for (int q = 0; q < NB; ++q) x = cfma(x, D[q * NB + r], Yb[q * LC + col]);
                W[((j0 + r) % WR) * LC + col] = x;
                if (col < ncol) B[(size_t)col * n + j0 + r] = x;
            }
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
    // squared moduli here, one square root per warp after the reduction: the
    // kernel is bound by the FP64 pipe (1/64 of the FP32 rate on this part),
    // and a modulus per element cost as much as the residual's products
    // (values of modulus up to about 1e150, far beyond any sample's)
    double2 acc[RES_LCH];
    double xm[RES_LCH];
#pragma unroll
    for (int l = 0; l < RES_LCH; ++l) {
        acc[l] = make_double2(0.0, 0.0);
        xm[l] = 0.0;
        if (i < n && l0 + l < L) {
            acc[l] = U[(size_t)(l0 + l) * n + i];
            const double2 x = Xp[(size_t)(l0 + l) * n + i];
            xm[l] = fma(x.x, x.x, x.y * x.y);
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
        double rv = fma(acc[l].x, acc[l].x, acc[l].y * acc[l].y), xv = xm[l];
        for (int off = 16; off; off >>= 1) {
            rv = fmax(rv, shfl_down(rv, off));
            xv = fmax(xv, shfl_down(xv, off));
        }
        if ((threadIdx.x & 31) == 0 && l0 + l < L) {
            atomic_max_nonneg(rmax + pt * L + l0 + l, sqrt(rv));
            atomic_max_nonneg(xmax + pt * L + l0 + l, sqrt(xv));
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

// D = (c64) S for a whole array
__global__ void narrow_all_kernel(float2 *__restrict__ D, const double2 *__restrict__ S, int64_t total) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        D[q] = to_c64(S[q]);
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

// ---- real path (real NEP at real points): real factor storage, complex S
// with zero imaginary parts (so the FP64 residual and the projection are
// shared with the complex path)

// X = (real part D, 0)
template <typename R>
__global__ void widen_real_kernel(double2 *__restrict__ X, const R *__restrict__ D, int64_t total) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        X[q] = make_double2((double)D[q], 0.0);
}

// D = Re R for points still refining
__global__ void narrow_real_kernel(float *__restrict__ D, const double2 *__restrict__ R, int64_t per_pt,
                                   const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip[pt]) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < per_pt;
         q += (int64_t)gridDim.x * blockDim.x)
        D[pt * per_pt + q] = (float)R[pt * per_pt + q].x;
}

// Re X += D for points still refining
__global__ void update_real_kernel(double2 *__restrict__ X, const float *__restrict__ D, int64_t per_pt,
                                   const int32_t *__restrict__ skip) {
    const int pt = blockIdx.y;
    if (skip[pt]) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < per_pt;
         q += (int64_t)gridDim.x * blockDim.x)
        X[pt * per_pt + q].x += (double)D[pt * per_pt + q];
}

// U = Re U (the real path's probe is real)
__global__ void real_part_kernel(double2 *__restrict__ U, int64_t total) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x)
        U[q].y = 0.0;
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
    // 8 columns per block of 256 threads
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((p.n + 7) / 8, 2048)), p.N);
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
static size_t solve_smem(const BandGeom &g) {
    const int WR = g.kl + g.ku + NB, PRM = NB + g.kl;
    const size_t gsz = std::max<size_t>((size_t)PRM * LC, (size_t)SV_WARPS * NB * LC);
    return sizeof(C) * ((size_t)WR * LC + gsz + (size_t)NB * SV_FCH + NB * NB + NB * LC) +
           sizeof(int) * PRM;
}

template <typename C, int NB, int LC>
static cudaError_t solve_dispatch(const C *ab, const int32_t *piv, const C *dinv, C *B,
                                  const BandGeom &g, int N, int n, int L, const int32_t *skip,
                                  cudaStream_t s) {
    const size_t smem = solve_smem<C, NB, LC>(g);
    const int limit = smem_optin_limit();
    if (smem > (size_t)limit) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<C, NB, LC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    if (e != cudaSuccess) return e;
    dim3 grid((L + LC - 1) / LC, N);
    band_solve_kernel<C, NB, LC><<<grid, SV_THREADS, smem, s>>>(ab, piv, dinv, B, n, g.kl, g.ku,
                                                                 g.ldab, L, skip);
    return cudaGetLastError();
}

// the right-hand-side chunk shrinks for wide bands so that the window fits
cudaError_t launch_band_solve_c64(const float2 *ab, const int32_t *piv, const float2 *dinv,
                                  float2 *B, const BandGeom &g, int N, int n, int L,
                                  const int32_t *skip, cudaStream_t s) {
    if (solve_smem<float2, NB_C64, 16>(g) <= 200 * 1024)
        return solve_dispatch<float2, NB_C64, 16>(ab, piv, dinv, B, g, N, n, L, skip, s);
    return solve_dispatch<float2, NB_C64, 8>(ab, piv, dinv, B, g, N, n, L, skip, s);
}
bool band_solve_fits_c128(const BandGeom &g) {
    return solve_smem<double2, NB_C128, 4>(g) <= (size_t)smem_optin_limit();
}
cudaError_t launch_band_solve_c128(const double2 *ab, const int32_t *piv, const double2 *dinv,
                                   double2 *B, const BandGeom &g, int N, int n, int L,
                                   const int32_t *skip, cudaStream_t s) {
    if (solve_smem<double2, NB_C128, 8>(g) <= 200 * 1024)
        return solve_dispatch<double2, NB_C128, 8>(ab, piv, dinv, B, g, N, n, L, skip, s);
    return solve_dispatch<double2, NB_C128, 4>(ab, piv, dinv, B, g, N, n, L, skip, s);
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
cudaError_t launch_narrow_all(float2 *D, const double2 *S, int64_t total, cudaStream_t s) {
    narrow_all_kernel<<<grid_for(total, 256), 256, 0, s>>>(D, S, total);
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

cudaError_t launch_broadcast_probe_r32(float *D, const double2 *U, int64_t nL, int N, cudaStream_t s) {
    broadcast_probe_kernel<float><<<grid_for(nL * N, 256), 256, 0, s>>>(D, U, nL, N);
    return cudaGetLastError();
}
cudaError_t launch_broadcast_probe_r64(double *D, const double2 *U, int64_t nL, int N, cudaStream_t s) {
    broadcast_probe_kernel<double><<<grid_for(nL * N, 256), 256, 0, s>>>(D, U, nL, N);
    return cudaGetLastError();
}
cudaError_t launch_widen_r32(double2 *X, const float *D, int64_t total, cudaStream_t s) {
    widen_real_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(X, D, total);
    return cudaGetLastError();
}
cudaError_t launch_widen_r64(double2 *X, const double *D, int64_t total, cudaStream_t s) {
    widen_real_kernel<double><<<grid_for(total, 256), 256, 0, s>>>(X, D, total);
    return cudaGetLastError();
}
cudaError_t launch_narrow_r32(float *D, const double2 *R, int64_t per_pt, int N, const int32_t *skip,
                              cudaStream_t s) {
    narrow_real_kernel<<<dim3(grid_for(per_pt, 256, 64), N), 256, 0, s>>>(D, R, per_pt, skip);
    return cudaGetLastError();
}
cudaError_t launch_update_r32(double2 *X, const float *D, int64_t per_pt, int N, const int32_t *skip,
                              cudaStream_t s) {
    update_real_kernel<<<dim3(grid_for(per_pt, 256, 64), N), 256, 0, s>>>(X, D, per_pt, skip);
    return cudaGetLastError();
}
cudaError_t launch_real_part(double2 *U, int64_t total, cudaStream_t s) {
    real_part_kernel<<<grid_for(total, 256), 256, 0, s>>>(U, total);
    return cudaGetLastError();
}
cudaError_t launch_band_solve_r32(const float *ab, const int32_t *piv, const float *dinv, float *B,
                                  const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s) {
    if (solve_smem<float, NB_C64, 16>(g) <= 200 * 1024)
        return solve_dispatch<float, NB_C64, 16>(ab, piv, dinv, B, g, N, n, L, skip, s);
    return solve_dispatch<float, NB_C64, 8>(ab, piv, dinv, B, g, N, n, L, skip, s);
}
cudaError_t launch_band_solve_r64(const double *ab, const int32_t *piv, const double *dinv, double *B,
                                  const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s) {
    if (solve_smem<double, NB_C128, 8>(g) <= 200 * 1024)
        return solve_dispatch<double, NB_C128, 8>(ab, piv, dinv, B, g, N, n, L, skip, s);
    return solve_dispatch<double, NB_C128, 4>(ab, piv, dinv, B, g, N, n, L, skip, s);
}

template cudaError_t launch_assemble<float>(float *, const BandGeom &, const DevProblem &, cudaStream_t);
template cudaError_t launch_assemble<double>(double *, const BandGeom &, const DevProblem &, cudaStream_t);
template cudaError_t launch_assemble<float2>(float2 *, const BandGeom &, const DevProblem &,
                                             cudaStream_t);
template cudaError_t launch_assemble<double2>(double2 *, const BandGeom &, const DevProblem &,
                                              cudaStream_t);

}  // namespace rsrr
