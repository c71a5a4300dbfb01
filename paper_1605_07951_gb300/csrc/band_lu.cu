// Batched banded LU with partial pivoting for RSRR step 2 (Section 3.3):
// the factorisation of every T(z_j), one CTA per sampling point.  The band
// storage is described in band.cu.
#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

constexpr int LU_THREADS = 512;
constexpr int LU_WARPS = LU_THREADS / 32;

// --------------------------------------------------------------------------
// Banded LU with partial pivoting, blocked by NB columns, one CTA per point.
//
// Panel (columns j0..j0+jb-1, rows j0..j0+pr-1, pr <= jb + kl): thread r owns
// panel row r in registers.  Per column: block-wide argmax of |re|+|im| over
// the candidate rows (first index on ties), the pivot row and the displaced
// row exchange through shared memory, then every row below scales its
// multiplier and updates its remaining panel entries.  Two barriers a column.
//
// Trailing columns c in [j0+jb, min(n, j0+jb+KV)) are updated in chunks of
// CW = 16*CB columns: U12 = L11^{-1} * (P A12) with an explicit inverse of
// the unit lower triangle L11 (computed once per panel), then
// A22 -= L21 * U12, accumulated in registers over row groups of 32 (RA of
// them cover the kl rows below the panel).  All reads of a chunk (through the
// row permutation of the panel) happen before any write of that chunk.
// --------------------------------------------------------------------------
template <typename C, int NB, int RA, int CB>
__global__ void __launch_bounds__(LU_THREADS, 1)
band_lu_kernel(C *__restrict__ ab_all, int32_t *__restrict__ piv_all,
               int32_t *__restrict__ info_all, C *__restrict__ dinv_all, int n, int kl, int ku,
               int ldab) {
    using R = typename real_of<C>::type;
    constexpr int CW = LU_WARPS * CB;
    constexpr int PRA = NB + 32 * RA;  // allocated panel rows (>= NB + kl)
    const int pt = blockIdx.x;
    C *ab = ab_all + (size_t)pt * ldab * n;
    int32_t *piv = piv_all + (size_t)pt * n;
    const int nblk = (n + NB - 1) / NB;
    // per block: L11^{-1} then U11^{-1}, both NB x NB column major
    C *dinv = dinv_all + (size_t)pt * nblk * 2 * NB * NB;
    const int KV = kl + ku;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *P = reinterpret_cast<C *>(smem_raw);  // [NB][PRA], column major
    C *Linv = P + NB * PRA;                  // [NB][NB+1], column major, padded
    C *Uinv = Linv + NB * (NB + 1);          // [NB][NB+1], column major, padded
    C *Ut = Uinv + NB * (NB + 1);            // [NB][CW]  (row t, col) at t*CW+col
    C *U2 = Ut + NB * CW;                    // [NB][CW]
    C *prow = U2 + NB * CW;                  // [2][NB]
    C *drow = prow + 2 * NB;                 // [2][NB]
    R *wval = reinterpret_cast<R *>(drow + 2 * NB);  // [2][LU_WARPS]
    int *widx = reinterpret_cast<int *>(wval + 2 * LU_WARPS);  // [2][LU_WARPS]
    int *perm = widx + 2 * LU_WARPS;         // [PRA]
    int *sw = perm + PRA;                    // [NB]

    for (int q = tid; q < NB * PRA; q += LU_THREADS) P[q] = czero<C>();
    int info = 0;
    __syncthreads();

    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = min(NB, n - j0);
        const int pr = min(n - j0, jb + kl);

        // ---------------- panel factorisation (rows in registers)
        C row[NB];
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) {
            row[cc] = czero<C>();
            if (tid < pr && cc < jb) {
                const int d = tid - cc;  // (j0 + tid) - (j0 + cc)
                if (d >= -KV && d < kl + NB) row[cc] = ab[(size_t)(j0 + cc) * ldab + KV + d];
            }
        }
#pragma unroll
        for (int cc = 0; cc < NB; ++cc) {
            if (cc < jb) {
                const int buf = cc & 1;
                const int rend = min(pr, cc + kl + 1);
                R v = (R)-1;
                int ix = 0x7fffffff;
                if (tid >= cc && tid < rend) { v = cabs1(row[cc]); ix = tid; }
#pragma unroll
                for (int off = 16; off; off >>= 1) {
                    const R ov = shfl_down(v, off);
                    const int oi = shfl_down(ix, off);
                    if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
                }
                if (lane == 0) { wval[buf * LU_WARPS + warp] = v; widx[buf * LU_WARPS + warp] = ix; }
                __syncthreads();
                R bv = wval[buf * LU_WARPS];
                int p = widx[buf * LU_WARPS];
#pragma unroll
                for (int w = 1; w < LU_WARPS; ++w) {
                    const R ov = wval[buf * LU_WARPS + w];
                    const int oi = widx[buf * LU_WARPS + w];
                    if (ov > bv || (ov == bv && oi < p)) { bv = ov; p = oi; }
                }
                if (tid == p) {
#pragma unroll
                    for (int c2 = 0; c2 < NB; ++c2) prow[buf * NB + c2] = row[c2];
                }
                if (tid == cc) {
#pragma unroll
                    for (int c2 = 0; c2 < NB; ++c2) drow[buf * NB + c2] = row[c2];
                }
                __syncthreads();
                if (tid == cc) {
#pragma unroll
                    for (int c2 = 0; c2 < NB; ++c2) row[c2] = prow[buf * NB + c2];
                } else if (tid == p) {
#pragma unroll
                    for (int c2 = 0; c2 < NB; ++c2) row[c2] = drow[buf * NB + c2];
                }
                const C pv = prow[buf * NB + cc];
                const bool nz = cnonzero(pv);
                if (tid > cc && tid < rend && nz) {
                    const C l = cmul(row[cc], crecip(pv));
                    row[cc] = l;
#pragma unroll
                    for (int c2 = cc + 1; c2 < NB; ++c2) row[c2] = cfms(row[c2], l, prow[buf * NB + c2]);
                }
                if (tid == 0) {
                    sw[cc] = p;
                    piv[j0 + cc] = j0 + p;
                    if (!nz && info == 0) info = j0 + cc + 1;
                }
            }
        }
        // panel -> shared (column major) and global
        if (tid < pr) {
#pragma unroll
            for (int cc = 0; cc < NB; ++cc) {
                if (cc < jb) {
                    P[cc * PRA + tid] = row[cc];
                    const int d = tid - cc;
                    if (d >= -KV && d < kl + NB) ab[(size_t)(j0 + cc) * ldab + KV + d] = row[cc];
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            for (int r = 0; r < pr; ++r) perm[r] = r;
            for (int cc = 0; cc < jb; ++cc) {
                const int p = sw[cc];
                const int t = perm[cc]; perm[cc] = perm[p]; perm[p] = t;
            }
        }
        if (warp == 1) {
            // column j = lane of L11^{-1}: x_i = [i == j] - sum_{t<i} L(i,t) x_t,
            // kept in shared memory (row stride NB + 1 avoids bank conflicts)
            const int j = lane;
            if (j < NB) {
                for (int i = 0; i < NB; ++i) {
                    C s = (i == j) ? cone<C>() : czero<C>();
                    for (int t = j; t < i; ++t) s = cfms(s, P[t * PRA + i], Linv[j * (NB + 1) + t]);
                    Linv[j * (NB + 1) + i] = (i < j || i >= jb || j >= jb) ? czero<C>() : s;
                }
            }
        } else if (warp == 2) {
            // column j = lane of U11^{-1}: x_j = 1/u_jj,
            // x_i = -(sum_{i<t<=j} u_it x_t) / u_ii for i = j-1 .. 0
            const int j = lane;
            if (j < NB) {
                for (int i = 0; i < NB; ++i) Uinv[j * (NB + 1) + i] = czero<C>();
                if (j < jb) {
                    Uinv[j * (NB + 1) + j] = crecip(P[j * PRA + j]);
                    for (int i = j - 1; i >= 0; --i) {
                        C s = czero<C>();
                        for (int t = i + 1; t <= j; ++t) s = cfma(s, P[t * PRA + i], Uinv[j * (NB + 1) + t]);
                        Uinv[j * (NB + 1) + i] = cmul(csub(czero<C>(), s), crecip(P[i * PRA + i]));
                    }
                }
            }
        }
        __syncthreads();
        {
            C *dst = dinv + (size_t)(j0 / NB) * 2 * NB * NB;
            for (int q = tid; q < 2 * NB * NB; q += LU_THREADS) {
                const int w = q / (NB * NB), e = q % (NB * NB), j = e / NB, i = e % NB;
                dst[q] = (w == 0 ? Linv : Uinv)[j * (NB + 1) + i];
            }
        }

        // ---------------- trailing update
        const int c_beg = j0 + jb;
        const int c_end = min(n, j0 + jb + KV);
        for (int c0 = c_beg; c0 < c_end; c0 += CW) {
            const int cw = min(CW, c_end - c0);
            // (1) all reads of the chunk: U rows into Ut, A22 into registers
            for (int o = tid; o < NB * CW; o += LU_THREADS) {
                const int t = o % NB, col = o / NB;
                C v = czero<C>();
                if (t < jb && col < cw) {
                    const int c = c0 + col;
                    const int d = j0 + perm[t] - c;
                    if (d >= -KV) v = ab[(size_t)c * ldab + KV + d];
                }
                Ut[t * CW + col] = v;
            }
            C acc[RA][CB];
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                const int r = jb + lane + 32 * a;
#pragma unroll
                for (int b = 0; b < CB; ++b) {
                    const int col = warp + LU_WARPS * b;
                    acc[a][b] = czero<C>();
                    if (r < pr && col < cw) {
                        const int c = c0 + col;
                        const int d = j0 + perm[r] - c;
                        if (d >= -KV) acc[a][b] = ab[(size_t)c * ldab + KV + d];
                    }
                }
            }
            __syncthreads();
            // (2) U12 = L11^{-1} Ut  -> U2 and global rows j0..j0+jb-1
            for (int o = tid; o < NB * CW; o += LU_THREADS) {
                const int t = o % NB, col = o / NB;
                C s = czero<C>();
#pragma unroll
                for (int q = 0; q < NB; ++q) s = cfma(s, Linv[q * (NB + 1) + t], Ut[q * CW + col]);
                U2[t * CW + col] = s;
                if (t < jb && col < cw) {
                    const int c = c0 + col;
                    const int d = j0 + t - c;
                    if (d >= -KV) ab[(size_t)c * ldab + KV + d] = s;
                }
            }
            __syncthreads();
            // (3) A22 -= L21 U12, rows j0+jb.., written at their (permuted) positions
#pragma unroll 4
            for (int q = 0; q < NB; ++q) {
                C uq[CB];
#pragma unroll
                for (int b = 0; b < CB; ++b) uq[b] = U2[q * CW + warp + LU_WARPS * b];
#pragma unroll
                for (int a = 0; a < RA; ++a) {
                    const C l = P[q * PRA + jb + lane + 32 * a];
#pragma unroll
                    for (int b = 0; b < CB; ++b) acc[a][b] = cfms(acc[a][b], l, uq[b]);
                }
            }
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                const int r = jb + lane + 32 * a;
#pragma unroll
                for (int b = 0; b < CB; ++b) {
                    const int col = warp + LU_WARPS * b;
                    if (r < pr && col < cw) {
                        const int c = c0 + col;
                        ab[(size_t)c * ldab + KV + (j0 + r - c)] = acc[a][b];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) info_all[pt] = info;
}

template <typename C, int NB, int RA, int CB>
static size_t lu_smem_bytes() {
    constexpr int CW = LU_WARPS * CB;
    constexpr int PRA = NB + 32 * RA;
    size_t b = sizeof(C) * ((size_t)NB * PRA + 2 * NB * (NB + 1) + 2 * NB * CW + 4 * NB);
    b += sizeof(typename real_of<C>::type) * 2 * LU_WARPS + sizeof(int) * (2 * LU_WARPS + PRA + NB);
    return b;
}

template <typename C, int NB, int RA, int CB>
static cudaError_t lu_dispatch(C *ab, int32_t *piv, int32_t *info, C *dinv, const BandGeom &g,
                               int N, int n, cudaStream_t s) {
    const size_t smem = lu_smem_bytes<C, NB, RA, CB>();
    cudaError_t e = cudaFuncSetAttribute(band_lu_kernel<C, NB, RA, CB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    band_lu_kernel<C, NB, RA, CB><<<N, LU_THREADS, smem, s>>>(ab, piv, info, dinv, n, g.kl, g.ku,
                                                               g.ldab);
    return cudaGetLastError();
}

template <typename C, int NB, int CB>
static cudaError_t lu_by_kl(C *ab, int32_t *piv, int32_t *info, C *dinv, const BandGeom &g, int N,
                            int n, cudaStream_t s) {
    const int kl = g.kl;
    if (kl <= 32) return lu_dispatch<C, NB, 1, CB>(ab, piv, info, dinv, g, N, n, s);
    if (kl <= 128) return lu_dispatch<C, NB, 4, CB>(ab, piv, info, dinv, g, N, n, s);
    if (kl <= 224) return lu_dispatch<C, NB, 7, CB>(ab, piv, info, dinv, g, N, n, s);
    return lu_dispatch<C, NB, 15, CB>(ab, piv, info, dinv, g, N, n, s);
}

#if !defined(RSRR_LU_ONLY) || RSRR_LU_ONLY == 64
cudaError_t launch_band_lu_c64(float2 *ab, int32_t *piv, int32_t *info, float2 *dinv,
                               const BandGeom &g, int N, int n, cudaStream_t s) {
    return lu_by_kl<float2, NB_C64, 4>(ab, piv, info, dinv, g, N, n, s);
}
#endif
#if !defined(RSRR_LU_ONLY) || RSRR_LU_ONLY == 128
cudaError_t launch_band_lu_c128(double2 *ab, int32_t *piv, int32_t *info, double2 *dinv,
                                const BandGeom &g, int N, int n, cudaStream_t s) {
    return lu_by_kl<double2, NB_C128, 1>(ab, piv, info, dinv, g, N, n, s);
}
#endif

}  // namespace rsrr
