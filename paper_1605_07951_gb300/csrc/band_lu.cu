// Batched banded LU with partial pivoting for RSRR step 2 (Section 4.3):
// the factorisation of every T(z_j).  The band storage is described in
// band.cu.  Two launch shapes share the same device routines and perform the
// same arithmetic on every element, in the same order:
//   band_lu_kernel          one CTA per sampling point;
//   band_lu_cluster_kernel  a cluster of two CTAs per point with a one-panel
//                           lookahead: CTA 0 updates the first chunk(s) of
//                           the trailing window (the first holds the next
//                           panel) and factors the next panel while CTA 1
//                           updates the rest of the window; one cluster
//                           barrier a panel.
// Global reads of the factor, pivots and block inverses bypass L1 (__ldcg):
// the two CTAs of a cluster sit on different SMs and read what the other
// wrote, and L1 is not coherent between SMs.
#include <algorithm>
#include <cooperative_groups.h>

#include "common.cuh"
#include "rsrr_internal.h"

namespace cg = cooperative_groups;

namespace rsrr {


// --------------------------------------------------------------------------
// Blocked by NB columns.
//
// Panel (columns j0..j0+jb-1, rows j0..j0+pr-1, pr <= jb + kl <= TH): thread r
// owns panel row r in registers.  Per column: block-wide argmax of |re|+|im| over
// the candidate rows (first index on ties), the pivot row and the displaced
// row exchange through shared memory, then every row below scales its
// multiplier and updates its remaining panel entries.  Two barriers a column.
//
// Trailing columns c in [j0+jb, min(n, j0+jb+KV)) are updated in chunks of
// CW = (TH/32)*CB columns: U12 = L11^{-1} * (P A12) with an explicit inverse of
// the unit lower triangle L11 (computed once per panel), then
// A22 -= L21 * U12, accumulated in registers over row groups of 32 (RA of
// them cover the kl rows below the panel).  All reads of a chunk (through the
// row permutation of the panel) happen before any write of that chunk.
// --------------------------------------------------------------------------
template <typename C, int NB, int RA, int CB, int TH>
struct LuSm {
    static constexpr int CW = (TH / 32) * CB;
    static constexpr int PRA = NB + 32 * RA;  // allocated panel rows (>= NB + kl)
    // padded strides: a column of P and a row of Ut / U2 start one element
    // apart in the banks, so the triangular inverses (a lane per column,
    // walking down the rows) and the transposing stores do not conflict
    static constexpr int PRS = PRA + 1;
    static constexpr int CWS = CW + 1;
    C *P;      // [NB][PRS], column major
    C *Linv;   // [NB][NB+1], column major, padded
    C *Uinv;   // [NB][NB+1]
    C *Ut;     // [NB][CWS]  (row t, col) at t*CWS+col
    C *U2;     // [NB][CWS]
    int *perm; // [PRA] position -> panel row
    int *pos;  // [PRA] panel row -> position (panel factorisation)
    int *sw;   // [NB]  pivots, as panel rows (factorisation) or positions (from piv)

    RSRR_DEV explicit LuSm(unsigned char *raw) {
        P = reinterpret_cast<C *>(raw);
        Linv = P + NB * PRS;
        Uinv = Linv + NB * (NB + 1);
        Ut = Uinv + NB * (NB + 1);
        U2 = Ut + NB * CWS;
        perm = reinterpret_cast<int *>(U2 + NB * CWS);
        pos = perm + PRA;
        sw = pos + PRA;
    }
    static size_t bytes() {
        return sizeof(C) * ((size_t)NB * PRS + 2 * NB * (NB + 1) + 2 * NB * CWS) + sizeof(int) * (2 * PRA + NB);
    }
};

// Factors the panel at column j0: the factored columns go to global memory
// and to sm.P, the pivots to piv, the composed row permutation to sm.perm,
// L11^{-1} and U11^{-1} to sm.Linv / sm.Uinv and to the block's dinv slot.
//
// The panel is factored in shared memory with its rows in their original
// order and the interchanges kept virtual: per column every warp that holds
// panel rows finds the pivot itself (argmax of |re|+|im| over the rows not
// yet pivots among the first cc + kl + 1, smallest row on ties; each lane
// keeps a bit mask of its rows that were pivots), so no barrier is needed
// to publish it; every other active row then forms its multiplier and
// updates its remaining panel entries against the pivot row.  One barrier a
// column.  A row's multiplier is stored after the barrier (a slower warp may
// still be reading the column for its pivot search).  At the end the
// interchanges are replayed in order, as positions (LAPACK's sequential
// swaps), for piv and sm.perm, and the rows are moved to their positions.
template <typename C, int NB, int RA, int CB, int TH>
RSRR_DEV void lu_panel(C *__restrict__ ab, int32_t *__restrict__ piv, C *__restrict__ dinv, int n,
                       int kl, int KV, int ldab, int j0, const LuSm<C, NB, RA, CB, TH> &sm, int &info) {
    using R = typename real_of<C>::type;
    constexpr int PRS = LuSm<C, NB, RA, CB, TH>::PRS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jb = min(NB, n - j0);
    const int pr = min(n - j0, jb + kl);
    // (1) rows j0 .. j0+pr-1, columns j0 .. j0+NB-1 into shared memory (zero
    // outside the band storage and beyond the last column)
    for (int q = tid; q < NB * pr; q += TH) {
        const int cc = q / pr, r = q % pr;
        const int d = r - cc;
        C v = czero<C>();
        if (cc < jb && d >= -KV && d < kl + NB) v = __ldcg(&ab[(size_t)(j0 + cc) * ldab + KV + d]);
        sm.P[cc * PRS + r] = v;
    }
    __syncthreads();
    // (2) the columns
    const bool scan = warp * 32 < pr;  // warps that hold panel rows
    unsigned dmask = 0;                // bit i: row lane + 32 i is a pivot already
    bool rdone = false;                // this thread's row is a pivot already
    C lprev = czero<C>();
    int cprev = -1;
    for (int cc = 0; cc < jb; ++cc) {
        if (cprev >= 0) {
            sm.P[cprev * PRS + tid] = lprev;
            cprev = -1;
        }
        if (scan) {
            const int rend = min(pr, cc + kl + 1);
            R v = (R)-1;
            int ix = 0x7fffffff;
            int i = 0;
            for (int r = lane; r < rend; r += 32, ++i) {
                if (!((dmask >> i) & 1u)) {
                    R a = cabs1(sm.P[cc * PRS + r]);
                    if (!(a >= (R)0)) a = (R)0;  // a NaN never wins, but a row is always chosen
                    if (a > v) { v = a; ix = r; }
                }
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) {
                const R ov = shfl_down(v, off);
                const int oi = shfl_down(ix, off);
                if (ov > v || (ov == v && oi < ix)) { v = ov; ix = oi; }
            }
            const int p = __shfl_sync(0xffffffffu, ix, 0);
            if ((p & 31) == lane) dmask |= 1u << (p >> 5);
            if (tid == p) rdone = true;
            const C pv = sm.P[cc * PRS + p];
            const bool nz = cnonzero(pv);
            if (tid < rend && !rdone && nz) {
                const C l = cmul(sm.P[cc * PRS + tid], crecip(pv));
                lprev = l;
                cprev = cc;
#pragma unroll 4
                for (int c2 = cc + 1; c2 < jb; ++c2)
                    sm.P[c2 * PRS + tid] = cfms(sm.P[c2 * PRS + tid], l, sm.P[c2 * PRS + p]);
            }
            if (tid == 0) {
                sm.sw[cc] = p;
                if (!nz && info == 0) info = j0 + cc + 1;
            }
        }
        __syncthreads();
    }
    if (cprev >= 0) sm.P[cprev * PRS + tid] = lprev;
    // (3) the interchanges as positions: piv and sm.perm (position -> row)
    for (int r = tid; r < pr; r += TH) {
        sm.perm[r] = r;
        sm.pos[r] = r;
    }
    __syncthreads();
    if (tid == 0) {
        for (int cc = 0; cc < jb; ++cc) {
            const int p = sm.sw[cc], pp = sm.pos[p], rc = sm.perm[cc];
            piv[j0 + cc] = j0 + pp;
            sm.perm[cc] = p;
            sm.perm[pp] = rc;
            sm.pos[p] = cc;
            sm.pos[rc] = pp;
        }
    }
    __syncthreads();
    // (4) rows to their positions, in shared memory and in the band storage
    constexpr int HALF = NB / 2;
    const int dpos = tid < pr ? sm.pos[tid] : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        C v[HALF];
#pragma unroll
        for (int c = 0; c < HALF; ++c) v[c] = tid < pr ? sm.P[(h * HALF + c) * PRS + tid] : czero<C>();
        __syncthreads();
        if (tid < pr) {
#pragma unroll
            for (int c = 0; c < HALF; ++c) {
                const int cc = h * HALF + c;
                sm.P[cc * PRS + dpos] = v[c];
                const int d = dpos - cc;
                if (cc < jb && d >= -KV && d < kl + NB) ab[(size_t)(j0 + cc) * ldab + KV + d] = v[c];
            }
        }
        __syncthreads();
    }
    if (warp == 1) {
        // column j = lane of L11^{-1}: x_i = [i == j] - sum_{t<i} L(i,t) x_t,
        // kept in shared memory (row stride NB + 1 avoids bank conflicts)
        const int j = lane;
        if (j < NB) {
            for (int i = 0; i < NB; ++i) {
                C s = (i == j) ? cone<C>() : czero<C>();
                for (int t = j; t < i; ++t) s = cfms(s, sm.P[t * PRS + i], sm.Linv[j * (NB + 1) + t]);
                sm.Linv[j * (NB + 1) + i] = (i < j || i >= jb || j >= jb) ? czero<C>() : s;
            }
        }
    } else if (warp == 2) {
        // column j = lane of U11^{-1}: x_j = 1/u_jj,
        // x_i = -(sum_{i<t<=j} u_it x_t) / u_ii for i = j-1 .. 0
        const int j = lane;
        if (j < NB) {
            for (int i = 0; i < NB; ++i) sm.Uinv[j * (NB + 1) + i] = czero<C>();
            if (j < jb) {
                sm.Uinv[j * (NB + 1) + j] = crecip(sm.P[j * PRS + j]);
                for (int i = j - 1; i >= 0; --i) {
                    C s = czero<C>();
                    for (int t = i + 1; t <= j; ++t) s = cfma(s, sm.P[t * PRS + i], sm.Uinv[j * (NB + 1) + t]);
                    sm.Uinv[j * (NB + 1) + i] = cmul(csub(czero<C>(), s), crecip(sm.P[i * PRS + i]));
                }
            }
        }
    }
    __syncthreads();
    C *dst = dinv + (size_t)(j0 / NB) * 2 * NB * NB;
    for (int q = tid; q < 2 * NB * NB; q += TH) {
        const int w = q / (NB * NB), e = q % (NB * NB), j = e / NB, i = e % NB;
        dst[q] = (w == 0 ? sm.Linv : sm.Uinv)[j * (NB + 1) + i];
    }
}

// What the trailing update of the panel at j0 needs, read back from global
// memory (written there by the CTA that factored it): the multipliers L21
// into sm.P, L11^{-1} into sm.Linv, and the composed permutation from piv.
template <typename C, int NB, int RA, int CB, int TH>
RSRR_DEV void lu_load_panel(const C *__restrict__ ab, const int32_t *__restrict__ piv,
                            const C *__restrict__ dinv, int n, int kl, int KV, int ldab, int j0,
                            const LuSm<C, NB, RA, CB, TH> &sm) {
    constexpr int PRA = LuSm<C, NB, RA, CB, TH>::PRA;
    constexpr int PRS = LuSm<C, NB, RA, CB, TH>::PRS;
    const int tid = threadIdx.x;
    const int jb = min(NB, n - j0);
    const int pr = min(n - j0, jb + kl);
    for (int q = tid; q < NB * PRA; q += TH) {
        const int cc = q / PRA, r = q % PRA;
        C v = czero<C>();
        if (cc < jb && r >= jb && r < pr) v = __ldcg(&ab[(size_t)(j0 + cc) * ldab + KV + (r - cc)]);
        sm.P[cc * PRS + r] = v;
    }
    const C *src = dinv + (size_t)(j0 / NB) * 2 * NB * NB;
    for (int q = tid; q < NB * NB; q += TH) {
        const int j = q / NB, i = q % NB;
        sm.Linv[j * (NB + 1) + i] = __ldcg(&src[q]);
    }
    // the panel's pivots, all in flight at once, then composed by one thread
    if (tid < jb) sm.sw[tid] = __ldcg(&piv[j0 + tid]) - j0;
    for (int r = tid; r < pr; r += TH) sm.perm[r] = r;
    __syncthreads();
    if (tid == 0) {
        for (int cc = 0; cc < jb; ++cc) {
            const int p = sm.sw[cc];
            const int t = sm.perm[cc]; sm.perm[cc] = sm.perm[p]; sm.perm[p] = t;
        }
    }
    __syncthreads();
}

// Trailing update of the panel at j0 over columns [c_lo, c_hi).
template <typename C, int NB, int RA, int CB, int TH>
RSRR_DEV void lu_update(C *__restrict__ ab, int n, int kl, int KV, int ldab, int j0, int c_lo,
                        int c_hi, const LuSm<C, NB, RA, CB, TH> &sm) {
    constexpr int CW = LuSm<C, NB, RA, CB, TH>::CW;
    constexpr int CWS = LuSm<C, NB, RA, CB, TH>::CWS;
    constexpr int PRS = LuSm<C, NB, RA, CB, TH>::PRS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int jb = min(NB, n - j0);
    const int pr = min(n - j0, jb + kl);
    for (int c0 = c_lo; c0 < c_hi; c0 += CW) {
        const int cw = min(CW, c_hi - c0);
        // (1) all reads of the chunk: U rows into Ut, A22 into registers
        for (int o = tid; o < NB * CW; o += TH) {
            const int t = o % NB, col = o / NB;
            C v = czero<C>();
            if (t < jb && col < cw) {
                const int c = c0 + col;
                const int d = j0 + sm.perm[t] - c;
                if (d >= -KV) v = __ldcg(&ab[(size_t)c * ldab + KV + d]);
            }
            sm.Ut[t * CWS + col] = v;
        }
        C acc[RA][CB];
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int r = jb + lane + 32 * a;
#pragma unroll
            for (int b = 0; b < CB; ++b) {
                const int col = warp + (TH / 32) * b;
                acc[a][b] = czero<C>();
                if (r < pr && col < cw) {
                    const int c = c0 + col;
                    const int d = j0 + sm.perm[r] - c;
                    if (d >= -KV) acc[a][b] = __ldcg(&ab[(size_t)c * ldab + KV + d]);
                }
            }
        }
        __syncthreads();
        // (2) U12 = L11^{-1} Ut  -> U2 and global rows j0..j0+jb-1
        // each thread two rows t and two columns of U12: half the shared
        // loads of one output per thread, the same sum order per element
        for (int o = tid; o < NB * CW / 4; o += TH) {
            const int t2 = 2 * (o % (NB / 2)), col2 = 2 * (o / (NB / 2));
            C s00 = czero<C>(), s10 = czero<C>(), s01 = czero<C>(), s11 = czero<C>();
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const C l0 = sm.Linv[q * (NB + 1) + t2], l1 = sm.Linv[q * (NB + 1) + t2 + 1];
                const C u0 = sm.Ut[q * CWS + col2], u1 = sm.Ut[q * CWS + col2 + 1];
                s00 = cfma(s00, l0, u0);
                s10 = cfma(s10, l1, u0);
                s01 = cfma(s01, l0, u1);
                s11 = cfma(s11, l1, u1);
            }
            const C sv[4] = {s00, s10, s01, s11};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int t = t2 + (e & 1), col = col2 + (e >> 1);
                sm.U2[t * CWS + col] = sv[e];
                if (t < jb && col < cw) {
                    const int c = c0 + col;
                    const int d = j0 + t - c;
                    if (d >= -KV) ab[(size_t)c * ldab + KV + d] = sv[e];
                }
            }
        }
        __syncthreads();
        // (3) A22 -= L21 U12, rows j0+jb.., written at their (permuted) positions
#pragma unroll 1
        for (int q = 0; q < NB; ++q) {
            C uq[CB];
#pragma unroll
            for (int b = 0; b < CB; ++b) uq[b] = sm.U2[q * CWS + warp + (TH / 32) * b];
#pragma unroll
            for (int a = 0; a < RA; ++a) {
                const C l = sm.P[q * PRS + jb + lane + 32 * a];
#pragma unroll
                for (int b = 0; b < CB; ++b) acc[a][b] = cfms(acc[a][b], l, uq[b]);
            }
        }
#pragma unroll
        for (int a = 0; a < RA; ++a) {
            const int r = jb + lane + 32 * a;
#pragma unroll
            for (int b = 0; b < CB; ++b) {
                const int col = warp + (TH / 32) * b;
                if (r < pr && col < cw) {
                    const int c = c0 + col;
                    ab[(size_t)c * ldab + KV + (j0 + r - c)] = acc[a][b];
                }
            }
        }
    }
    __syncthreads();
}

// One CTA per point: panel, then the whole trailing window, panel by panel.
template <typename C, int NB, int RA, int CB, int TH>
__global__ void __launch_bounds__(TH, 1)
band_lu_kernel(C *__restrict__ ab_all, int32_t *__restrict__ piv_all,
               int32_t *__restrict__ info_all, C *__restrict__ dinv_all, int n, int kl, int ku,
               int ldab) {
    const int pt = blockIdx.x;
    C *ab = ab_all + (size_t)pt * ldab * n;
    int32_t *piv = piv_all + (size_t)pt * n;
    const int nblk = (n + NB - 1) / NB;
    // per block: L11^{-1} then U11^{-1}, both NB x NB column major
    C *dinv = dinv_all + (size_t)pt * nblk * 2 * NB * NB;
    const int KV = kl + ku;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LuSm<C, NB, RA, CB, TH> sm(smem_raw);
    for (int q = threadIdx.x; q < NB * LuSm<C, NB, RA, CB, TH>::PRS; q += TH) sm.P[q] = czero<C>();
    int info = 0;
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = min(NB, n - j0);
        lu_panel<C, NB, RA, CB, TH>(ab, piv, dinv, n, kl, KV, ldab, j0, sm, info);
        lu_update<C, NB, RA, CB, TH>(ab, n, kl, KV, ldab, j0, j0 + jb, min(n, j0 + jb + KV), sm);
    }
    if (threadIdx.x == 0) info_all[pt] = info;
}

// A cluster of two CTAs per point.  Iteration of panel j0 (factored and
// published in global memory before the iteration starts):
//   CTA 0: update the first chunk(s) of columns [j0+jb, j0+jb+KV) -- the
//          first holds the next panel -- then factor the next panel;
//   CTA 1: load the panel's multipliers, L11^{-1} and permutation from global
//          memory, update the remaining chunks;
//   cluster barrier (release/acquire; every thread of both CTAs).
// The barrier orders CTA 1's writes of a panel before CTA 0 reads them as
// the next panel's columns, and CTA 0's factored panel before CTA 1 loads
// it.  Both CTAs run the same number of barriers: one before the loop, one
// per panel, with no exit in between.
template <typename C, int NB, int RA, int CB, int TH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TH, 1)
band_lu_cluster_kernel(C *__restrict__ ab_all, int32_t *__restrict__ piv_all,
                       int32_t *__restrict__ info_all, C *__restrict__ dinv_all, int n, int kl,
                       int ku, int ldab) {
    constexpr int CW = LuSm<C, NB, RA, CB, TH>::CW;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const int pt = blockIdx.x / 2;
    C *ab = ab_all + (size_t)pt * ldab * n;
    int32_t *piv = piv_all + (size_t)pt * n;
    const int nblk = (n + NB - 1) / NB;
    C *dinv = dinv_all + (size_t)pt * nblk * 2 * NB * NB;
    const int KV = kl + ku;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LuSm<C, NB, RA, CB, TH> sm(smem_raw);
    for (int q = threadIdx.x; q < NB * LuSm<C, NB, RA, CB, TH>::PRS; q += TH) sm.P[q] = czero<C>();
    int info = 0;
    __syncthreads();
    if (rank == 0) lu_panel<C, NB, RA, CB, TH>(ab, piv, dinv, n, kl, KV, ldab, 0, sm, info);
    __threadfence();
    cluster.sync();
    for (int j0 = 0; j0 < n; j0 += NB) {
        const int jb = min(NB, n - j0);
        const int c_beg = j0 + jb, c_end = min(n, j0 + jb + KV);
        // CTA 0 takes the first `s` chunks (the first holds the next panel):
        // its panel costs about two chunks of update, so s = (chunks - 2) / 2
        // balances the two CTAs
        const int nch = (c_end - c_beg + CW - 1) / CW;
        const int c_split = min(c_end, c_beg + max(1, (nch - 2) / 2) * CW);
        if (rank == 0) {
            lu_update<C, NB, RA, CB, TH>(ab, n, kl, KV, ldab, j0, c_beg, c_split, sm);
            if (c_beg < n) lu_panel<C, NB, RA, CB, TH>(ab, piv, dinv, n, kl, KV, ldab, c_beg, sm, info);
        } else {
            lu_load_panel<C, NB, RA, CB, TH>(ab, piv, dinv, n, kl, KV, ldab, j0, sm);
            lu_update<C, NB, RA, CB, TH>(ab, n, kl, KV, ldab, j0, c_split, c_end, sm);
        }
        __threadfence();
        cluster.sync();
    }
    if (rank == 0 && threadIdx.x == 0) info_all[pt] = info;
}

// Many problems of uneven size in one persistent launch: every CTA takes
// the next (problem, point) task from a device counter (the host orders the
// tasks longest first) and factors it exactly as band_lu_kernel would, so the
// factors are bitwise those of the one-CTA kernel.  The instance covers the
// widest lower bandwidth of the batch (kl <= 32 RA).
template <typename C, int NB, int RA, int CB, int TH>
__global__ void __launch_bounds__(TH, 1)
band_lu_grouped_kernel(const LuTask *__restrict__ tasks, int ntasks, int *__restrict__ next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LuSm<C, NB, RA, CB, TH> sm(smem_raw);
    __shared__ int s_task;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(next, 1);
        __syncthreads();
        const int t = s_task;
        __syncthreads();
        if (t >= ntasks) break;
        const LuTask tk = tasks[t];
        C *ab = static_cast<C *>(tk.ab);
        C *dinv = static_cast<C *>(tk.dinv);
        const int n = tk.n, kl = tk.kl, KV = tk.kl + tk.ku, ldab = tk.ldab;
        for (int q = threadIdx.x; q < NB * LuSm<C, NB, RA, CB, TH>::PRS; q += TH) sm.P[q] = czero<C>();
        int info = 0;
        __syncthreads();
        for (int j0 = 0; j0 < n; j0 += NB) {
            const int jb = min(NB, n - j0);
            lu_panel<C, NB, RA, CB, TH>(ab, tk.piv, dinv, n, kl, KV, ldab, j0, sm, info);
            lu_update<C, NB, RA, CB, TH>(ab, n, kl, KV, ldab, j0, j0 + jb, min(n, j0 + jb + KV), sm);
        }
        if (threadIdx.x == 0) *tk.info = info;
        __syncthreads();
    }
}

template <typename C, int NB, int RA, int CB, int TH>
static cudaError_t lu_grouped(const LuTask *tasks, int ntasks, int *next, cudaStream_t s) {
    const size_t smem = LuSm<C, NB, RA, CB, TH>::bytes();
    cudaError_t e = cudaFuncSetAttribute(band_lu_grouped_kernel<C, NB, RA, CB, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    band_lu_grouped_kernel<C, NB, RA, CB, TH><<<std::max(1, std::min(ntasks, sms)), TH, smem, s>>>(tasks, ntasks,
                                                                                                   next);
    return cudaGetLastError();
}

template <typename C, int NB, int CB512>
static cudaError_t grouped_by_kl(const LuTask *tasks, int ntasks, int kl_max, int *next, cudaStream_t s) {
    constexpr int CB256 = 2 * CB512;
    if (kl_max <= 32) return lu_grouped<C, NB, 1, CB256, 256>(tasks, ntasks, next, s);
    if (kl_max <= 128) return lu_grouped<C, NB, 4, CB256, 256>(tasks, ntasks, next, s);
    if (kl_max <= 224) return lu_grouped<C, NB, 7, CB256, 256>(tasks, ntasks, next, s);
    return lu_grouped<C, NB, 15, CB512, 512>(tasks, ntasks, next, s);
}

template <typename C, int NB, int RA, int CB, int TH>
static cudaError_t lu_dispatch(C *ab, int32_t *piv, int32_t *info, C *dinv, const BandGeom &g,
                               int N, int n, bool cluster, cudaStream_t s) {
    const size_t smem = LuSm<C, NB, RA, CB, TH>::bytes();
    if (cluster) {
        cudaError_t e = cudaFuncSetAttribute(band_lu_cluster_kernel<C, NB, RA, CB, TH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        band_lu_cluster_kernel<C, NB, RA, CB, TH><<<2 * N, TH, smem, s>>>(ab, piv, info, dinv, n, g.kl,
                                                                              g.ku, g.ldab);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(band_lu_kernel<C, NB, RA, CB, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    band_lu_kernel<C, NB, RA, CB, TH><<<N, TH, smem, s>>>(ab, piv, info, dinv, n, g.kl, g.ku, g.ldab);
    return cudaGetLastError();
}

// Panel rows need one thread each: 256 threads cover kl <= 224 (more
// registers per thread for the trailing update), 512 threads the wider bands.
// The chunk width CW = (threads / 32) * CB is the same in both, so every
// element is computed the same way.
template <typename C, int NB, int CB512>
static cudaError_t lu_by_kl(C *ab, int32_t *piv, int32_t *info, C *dinv, const BandGeom &g, int N,
                            int n, bool cluster, cudaStream_t s) {
    const int kl = g.kl;
    constexpr int CB256 = 2 * CB512;
    if (kl <= 32) return lu_dispatch<C, NB, 1, CB256, 256>(ab, piv, info, dinv, g, N, n, cluster, s);
    if (kl <= 128) return lu_dispatch<C, NB, 4, CB256, 256>(ab, piv, info, dinv, g, N, n, cluster, s);
    // 512 threads for the single-precision types: sixteen warps hide the
    // latencies of the trailing update better than eight (measured 11% on the
    // full-size grid problem at half-bandwidth 200); same chunk width
    if (kl <= 224 && sizeof(C) <= 8) return lu_dispatch<C, NB, 7, CB512, 512>(ab, piv, info, dinv, g, N, n, cluster, s);
    if (kl <= 224) return lu_dispatch<C, NB, 7, CB256, 256>(ab, piv, info, dinv, g, N, n, cluster, s);
    return lu_dispatch<C, NB, 15, CB512, 512>(ab, piv, info, dinv, g, N, n, cluster, s);
}

#if !defined(RSRR_LU_ONLY) || RSRR_LU_ONLY == 64
cudaError_t launch_band_lu_grouped_c64(const LuTask *tasks, int ntasks, int kl_max, int *next, cudaStream_t s) {
    if (kl_max > KL_MAX) return cudaErrorInvalidValue;
    return grouped_by_kl<float2, NB_C64, 4>(tasks, ntasks, kl_max, next, s);
}
cudaError_t launch_band_lu_c64(float2 *ab, int32_t *piv, int32_t *info, float2 *dinv,
                               const BandGeom &g, int N, int n, cudaStream_t s, bool cluster) {
    return lu_by_kl<float2, NB_C64, 4>(ab, piv, info, dinv, g, N, n, cluster, s);
}
#endif
// real factors (real NEP at real points): RSRR_LU_ONLY = 32 (float), 65 (double)
#if !defined(RSRR_LU_ONLY) || RSRR_LU_ONLY == 32
cudaError_t launch_band_lu_r32(float *ab, int32_t *piv, int32_t *info, float *dinv, const BandGeom &g, int N,
                               int n, cudaStream_t s, bool cluster) {
    return lu_by_kl<float, NB_C64, 4>(ab, piv, info, dinv, g, N, n, cluster, s);
}
#endif
#if !defined(RSRR_LU_ONLY) || RSRR_LU_ONLY == 65
cudaError_t launch_band_lu_r64(double *ab, int32_t *piv, int32_t *info, double *dinv, const BandGeom &g, int N,
                               int n, cudaStream_t s, bool cluster) {
    return lu_by_kl<double, NB_C128, 1>(ab, piv, info, dinv, g, N, n, cluster, s);
}
#endif
#if !defined(RSRR_LU_ONLY) || RSRR_LU_ONLY == 128
cudaError_t launch_band_lu_grouped_c128(const LuTask *tasks, int ntasks, int kl_max, int *next, cudaStream_t s) {
    if (kl_max > KL_MAX) return cudaErrorInvalidValue;
    return grouped_by_kl<double2, NB_C128, 1>(tasks, ntasks, kl_max, next, s);
}
cudaError_t launch_band_lu_c128(double2 *ab, int32_t *piv, int32_t *info, double2 *dinv,
                                const BandGeom &g, int N, int n, cudaStream_t s, bool cluster) {
    return lu_by_kl<double2, NB_C128, 1>(ab, piv, info, dinv, g, N, n, cluster, s);
}
#endif

}  // namespace rsrr
