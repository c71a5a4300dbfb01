// Streaming banded solve with the factors of band_lu_kernel: X = (P L U)^{-1} B
// for every sampling point (Section 4.3's X_j = T(z_j)^{-1} U), one CTA per
// (point, chunk of LC right-hand sides).
//
// Forward, block by block (NB rows): the block's composed row permutation
// (precomputed by block_perm_kernel as at most 2 NB (position, source)
// pairs) is applied to the shared-memory window, y = L11^{-1} (P b)_top,
// and the rows below are updated, b_below -= L21 y.  Backward, from the last
// block: x = U11^{-1} y_block, then the rows above are updated,
// y_above -= U_above x (the same column-panel form as the forward pass).
//
// The factor panels (L21 below / U above a block, one contiguous run per
// column in the band layout) stream through a ring of shared-memory slots
// by cp.async, S2_DIST units ahead of the arithmetic; a unit is one chunk
// of S2_RC panel rows of one block (plus, for a block's first unit, its
// diagonal-block inverse, its permutation pairs and the window rows that
// enter with it).  Runs start at any 8-byte boundary: each column copies
// the 16-byte-aligned superset and reads from its offset.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

constexpr int S2_THREADS = 512;
// Two unit shapes: RC = 256 panel rows per unit with two ring slots (8
// right-hand sides of one row per thread: fewer shared-memory loads per FMA),
// used when it fits in shared memory, else RC = 128 with three slots.

// ---------------------------------------------------------------------------
// Composed permutation of each block: the LU swaps row j0+cc with piv[j0+cc]
// for cc = 0..jb-1 in order; position r of the block's window (rows j0 ..
// j0+pr-1) then holds original row j0 + perm[r].  Output: 2 NB entries per
// block, (r << 16) | perm[r] for every r with perm[r] != r, then -1.
// One warp per (point, block).
// ---------------------------------------------------------------------------
constexpr int BP_WARPS = 8;
constexpr int BP_MAXR = KL_MAX + 32;

__global__ void block_perm_kernel(int32_t *__restrict__ bperm, const int32_t *__restrict__ piv_all,
                                  int n, int kl, int NB, int nblk, int N) {
    __shared__ int sp[BP_WARPS][BP_MAXR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int PAIRS = 2 * NB;
    const int64_t total = (int64_t)N * nblk;
    for (int64_t task = (int64_t)blockIdx.x * BP_WARPS + w; task < total;
         task += (int64_t)gridDim.x * BP_WARPS) {
        const int pt = (int)(task / nblk), j = (int)(task % nblk);
        const int j0 = j * NB;
        const int jb = min(NB, n - j0);
        const int pr = min(n - j0, jb + kl);
        int *perm = sp[w];
        for (int r = lane; r < pr; r += 32) perm[r] = r;
        __syncwarp();
        if (lane == 0) {
            const int32_t *piv = piv_all + (size_t)pt * n + j0;
            for (int cc = 0; cc < jb; ++cc) {
                int p = piv[cc] - j0;
                if (p < cc || p >= pr) p = cc;  // out-of-range pivots never come from the LU
                const int t = perm[cc];
                perm[cc] = perm[p];
                perm[p] = t;
            }
        }
        __syncwarp();
        int32_t *out = bperm + (size_t)task * PAIRS;
        int cnt = 0;
        for (int r0 = 0; r0 < pr; r0 += 32) {
            const int r = r0 + lane;
            const bool moved = r < pr && perm[r] != r;
            const unsigned m = __ballot_sync(0xffffffffu, moved);
            const int pos = cnt + __popc(m & ((1u << lane) - 1u));
            if (moved && pos < PAIRS) out[pos] = (r << 16) | perm[r];
            cnt += __popc(m);
        }
        for (int e = cnt + lane; e < PAIRS; e += 32) out[e] = -1;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
RSRR_DEV void s2_cp16(unsigned saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g));
}
RSRR_DEV void s2_cp8(unsigned saddr, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr), "l"(g));
}
RSRR_DEV void s2_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
RSRR_DEV void s2_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

template <typename C> RSRR_DEV void s2_cp_elem(unsigned saddr, const C *g);
template <> RSRR_DEV void s2_cp_elem<float2>(unsigned saddr, const float2 *g) { s2_cp8(saddr, g); }
template <> RSRR_DEV void s2_cp_elem<double2>(unsigned saddr, const double2 *g) { s2_cp16(saddr, g); }
RSRR_DEV void s2_cp4(unsigned saddr, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(g));
}
template <> RSRR_DEV void s2_cp_elem<float>(unsigned saddr, const float *g) { s2_cp4(saddr, g); }
template <> RSRR_DEV void s2_cp_elem<double>(unsigned saddr, const double *g) { s2_cp8(saddr, g); }

template <typename C, int NB, int LC, int S2_RC, int S2_NSLOT>
struct S2Layout {
    static constexpr int E16 = 16 / (int)sizeof(C);          // elements per 16 bytes
    static constexpr int PLD = S2_RC + E16;                   // panel column stride (elements)
    static constexpr int MAXCH = PLD * (int)sizeof(C) / 16;   // 16-byte copies per column
    static constexpr int PAIRS = 2 * NB;
    static constexpr size_t D_BYTES = sizeof(C) * NB * NB;
    static constexpr size_t P_BYTES = 4 * PAIRS;
    static constexpr size_t PAN_BYTES = sizeof(C) * NB * PLD;
    static constexpr size_t SLOT = D_BYTES + P_BYTES + PAN_BYTES;
    static constexpr int WLD = LC + 1;  // window row stride: rows of a warp fall in different banks
    static RSRR_HD size_t w_bytes(int WR) { return ((sizeof(C) * (size_t)WR * WLD + 15) / 16) * 16; }
    static size_t smem(int WR) {
        return w_bytes(WR) + S2_NSLOT * SLOT + sizeof(C) * NB * LC + sizeof(C) * (size_t)PAIRS * LC;
    }
};

// block geometry shared by producer and consumer
struct S2Blk {
    int j0, jb, pr;
};
RSRR_DEV S2Blk s2_blk(int j, int n, int NB, int kl) {
    S2Blk b;
    b.j0 = j * NB;
    b.jb = min(NB, n - b.j0);
    b.pr = min(n - b.j0, b.jb + kl);
    return b;
}
// panel rows of a block: forward rows [jb, pr) below j0, backward the
// min(KV, j0) rows above j0
RSRR_DEV int s2_rows(int phase, const S2Blk &b, int KV) {
    return phase == 0 ? b.pr - b.jb : min(KV, b.j0);
}
template <int S2_RC>
RSRR_DEV int s2_units(int phase, const S2Blk &b, int KV) {
    return max(1, (s2_rows(phase, b, KV) + S2_RC - 1) / S2_RC);
}

template <typename C, int NB, int LC, int S2_RC, int S2_NSLOT>
__global__ void __launch_bounds__(S2_THREADS, 1)
band_solve2_kernel(const C *__restrict__ ab_all, const int32_t *__restrict__ bperm_all,
                   const C *__restrict__ dinv_all, C *__restrict__ B_all, int n, int kl, int ku,
                   int ldab, int L, int WR, const int32_t *__restrict__ skip,
                   const int32_t *__restrict__ gate, int gate_want) {
    using LY = S2Layout<C, NB, LC, S2_RC, S2_NSLOT>;
    // a gated launch runs only if the gate word holds gate_want (one of the
    // two shapes of a refinement sweep, chosen on the device)
    if (gate && __ldg(gate) != gate_want) return;
    constexpr int S2_DIST = S2_NSLOT - 1;
    constexpr int E16 = LY::E16, PLD = LY::PLD, MAXCH = LY::MAXCH, PAIRS = LY::PAIRS;
    constexpr int WLD = LY::WLD;
    constexpr int CG = LC * S2_RC / S2_THREADS;  // right-hand sides per thread in an update
    static_assert(CG >= 1 && LC % CG == 0, "update mapping");
    const int pt = blockIdx.y;
    if (skip && skip[pt]) return;
    const int col0 = blockIdx.x * LC;
    const int ncol = min(LC, L - col0);
    const int nblk = (n + NB - 1) / NB;
    const int KV = kl + ku;
    const size_t pbase = (size_t)pt * ldab * n;  // element offset of the point's factor
    const C *ab = ab_all + pbase;
    const C *dinv = dinv_all + (size_t)pt * nblk * 2 * NB * NB;
    const int32_t *bperm = bperm_all + (size_t)pt * nblk * PAIRS;
    C *B = B_all + (size_t)pt * L * n + (size_t)col0 * n;
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char s2_smem[];
    C *W = reinterpret_cast<C *>(s2_smem);                       // [WR][WLD]
    unsigned char *slots = s2_smem + LY::w_bytes(WR);             // S2_NSLOT x SLOT
    C *Yb = reinterpret_cast<C *>(slots + S2_NSLOT * LY::SLOT);  // [NB][LC]
    C *Gp = Yb + NB * LC;                                          // [LC][PAIRS]
    const unsigned s_base = (unsigned)__cvta_generic_to_shared(s2_smem);
    const unsigned s_slots = s_base + (unsigned)LY::w_bytes(WR);

    for (int phase = 0; phase < 2; ++phase) {
        // unit cursors: producer p*, consumer c*
        int pj = phase == 0 ? 0 : nblk - 1, pk = 0, pu = 0;
        bool pdone = false;
        auto advance = [&](int &j, int &k) -> bool {  // false at the end of the phase
            const S2Blk b = s2_blk(j, n, NB, kl);
            if (++k < s2_units<S2_RC>(phase, b, KV)) return true;
            k = 0;
            j += phase == 0 ? 1 : -1;
            return phase == 0 ? j < nblk : j >= 0;
        };
        auto issue = [&]() {
            if (pdone) { s2_commit(); return; }
            const S2Blk b = s2_blk(pj, n, NB, kl);
            const unsigned slot = s_slots + (unsigned)((pu % S2_NSLOT) * LY::SLOT);
            if (pk == 0) {
                // diagonal-block inverse: L11^{-1} (forward) or U11^{-1} (backward)
                const C *src = dinv + ((size_t)pj * 2 + phase) * NB * NB;
                for (int q = tid; q < (int)(LY::D_BYTES / 16); q += S2_THREADS)
                    s2_cp16(slot + q * 16, reinterpret_cast<const unsigned char *>(src) + q * 16);
                if (phase == 0)
                    for (int q = tid; q < (int)(LY::P_BYTES / 16); q += S2_THREADS)
                        s2_cp16(slot + (unsigned)LY::D_BYTES + q * 16,
                                reinterpret_cast<const unsigned char *>(bperm + (size_t)pj * PAIRS) + q * 16);
                // window rows entering with this block
                int r0, r1;
                if (phase == 0) {
                    r0 = pj == 0 ? 0 : b.j0 + kl;
                    r1 = min(n, b.j0 + b.jb + kl);
                } else {
                    r0 = max(0, b.j0 - KV);
                    r1 = pj == nblk - 1 ? n : max(0, b.j0 + NB - KV);
                }
                // rows r0 .. r1-1 (fewer than WR) in 32-row by 16-column passes
                const int nr = max(0, r1 - r0);
                const int w0 = r0 % WR;
                for (int rb = 0; rb < nr; rb += 32)
                    for (int cb = 0; cb < LC; cb += S2_THREADS / 32) {
                        const int rr = rb + (tid & 31), col = cb + (tid >> 5);
                        if (rr >= nr || col >= LC) continue;
                        int wrow = w0 + rr;
                        if (wrow >= WR) wrow -= WR;
                        C *dst = W + (size_t)wrow * WLD + col;
                        if (col < ncol)
                            s2_cp_elem<C>((unsigned)__cvta_generic_to_shared(dst), B + (size_t)col * n + r0 + rr);
                        else
                            *dst = czero<C>();
                    }
            }
            const int rows = s2_rows(phase, b, KV);
            const int ra = pk * S2_RC;
            if (ra < rows) {
                const int len = min(S2_RC, rows - ra);
                const unsigned pan = slot + (unsigned)(LY::D_BYTES + LY::P_BYTES);
                for (int o = tid; o < b.jb * MAXCH; o += S2_THREADS) {
                    const int t = o / MAXCH, q = o % MAXCH;
                    const int c = b.j0 + t;
                    // first panel row: forward row j0 + jb + ra, backward row j0 - rows + ra
                    const int i = phase == 0 ? b.j0 + b.jb + ra : b.j0 - rows + ra;
                    const int64_t s = (int64_t)c * ldab + KV + i - c;  // element offset in the point
                    const int off = (int)((pbase + (size_t)s) % E16);
                    if (q * E16 < len + off)
                        s2_cp16(pan + (unsigned)((t * PLD) * sizeof(C) + q * 16),
                                reinterpret_cast<const unsigned char *>(ab + s - off) + q * 16);
                }
            }
            s2_commit();
            ++pu;
            if (!advance(pj, pk)) pdone = true;
        };

        for (int d = 0; d < S2_DIST; ++d) issue();
        int cj = phase == 0 ? 0 : nblk - 1, ck = 0, cu = 0;
        for (;;) {
            s2_wait<S2_DIST - 1>();
            __syncthreads();
            issue();
            const S2Blk b = s2_blk(cj, n, NB, kl);
            const unsigned char *slot = slots + (cu % S2_NSLOT) * LY::SLOT;
            const C *D = reinterpret_cast<const C *>(slot);
            const int32_t *pairs = reinterpret_cast<const int32_t *>(slot + LY::D_BYTES);
            const C *P = reinterpret_cast<const C *>(slot + LY::D_BYTES + LY::P_BYTES);
            // window row of the block's first row: a multiple of NB at most
            // WR - NB, so the block's rows jb0 .. jb0+NB-1 do not wrap; rows
            // below it (offsets < kl + NB <= WR) wrap at most once
            const int jb0 = b.j0 % WR;
            auto wrow = [&](int off) { const int r = jb0 + off; return r >= WR ? r - WR : r; };
            if (ck == 0) {
                if (phase == 0) {
                    // composed permutation of the block's window
                    for (int o = tid; o < PAIRS * LC; o += S2_THREADS) {
                        const int e = o % PAIRS, col = o / PAIRS;
                        const int pr = pairs[e];
                        if (pr >= 0) Gp[col * PAIRS + e] = W[(size_t)wrow(pr & 0xFFFF) * WLD + col];
                    }
                    __syncthreads();
                    for (int o = tid; o < PAIRS * LC; o += S2_THREADS) {
                        const int e = o % PAIRS, col = o / PAIRS;
                        const int pr = pairs[e];
                        if (pr >= 0) W[(size_t)wrow(pr >> 16) * WLD + col] = Gp[col * PAIRS + e];
                    }
                    __syncthreads();
                }
                // y = L11^{-1} (P b)_top  or  x = U11^{-1} y_block
                for (int o = tid; o < NB * LC; o += S2_THREADS) {
                    const int col = o % LC, r = o / LC;
                    C v = czero<C>();
                    if (r < b.jb) {
                        const C *Wb = W + (size_t)jb0 * WLD + col;
#pragma unroll 8
                        for (int t = 0; t < b.jb; ++t)
                            v = cfma(v, D[t * NB + r], Wb[(size_t)t * WLD]);
                        if (col < ncol) B[(size_t)col * n + b.j0 + r] = v;
                    }
                    Yb[r * LC + col] = v;
                }
                __syncthreads();
            }
            // update of one panel chunk: W[rows] -= P Yb
            const int rows = s2_rows(phase, b, KV);
            const int ra = ck * S2_RC;
            if (ra < rows) {
                const int len = min(S2_RC, rows - ra);
                const int rr = tid % S2_RC, cg = tid / S2_RC;
                if (rr < len) {
                    const int i = phase == 0 ? b.j0 + b.jb + ra + rr : b.j0 - rows + ra + rr;
                    const int i0 = phase == 0 ? b.j0 + b.jb + ra : b.j0 - rows + ra;
                    C *wr = W + (size_t)(i % WR) * WLD + cg * CG;
                    C acc[CG];
#pragma unroll
                    for (int c = 0; c < CG; ++c) acc[c] = wr[c];
                    // backward: U(i, j0+t) lies in the band only for t <= i + KV - j0
                    const int tmax = phase == 0 ? b.jb : min(b.jb, i + KV - b.j0 + 1);
                    const int64_t s0 = (int64_t)b.j0 * ldab + KV + i0 - b.j0;  // run start of t = 0
#pragma unroll 4
                    for (int t = 0; t < tmax; ++t) {
                        const int off = (int)((pbase + (size_t)(s0 + (int64_t)t * (ldab - 1))) % E16);
                        const C l = P[t * PLD + off + rr];
                        const C *y = Yb + t * LC + cg * CG;
#pragma unroll
                        for (int c = 0; c < CG; ++c) acc[c] = cfms(acc[c], l, y[c]);
                    }
#pragma unroll
                    for (int c = 0; c < CG; ++c) wr[c] = acc[c];
                }
            }
            ++cu;
            if (!advance(cj, ck)) break;
        }
        s2_wait<0>();
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
static int bp_grid(int64_t tasks) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((tasks + BP_WARPS - 1) / BP_WARPS, 152 * 8));
}

cudaError_t launch_block_perm(int32_t *bperm, const int32_t *piv, int n, int kl, int nb, int N,
                              cudaStream_t s) {
    if (kl + nb > BP_MAXR) return cudaErrorInvalidValue;
    const int nblk = (n + nb - 1) / nb;
    block_perm_kernel<<<bp_grid((int64_t)N * nblk), BP_WARPS * 32, 0, s>>>(bperm, piv, n, kl, nb, nblk, N);
    return cudaGetLastError();
}

// window rows: every row live at once, rounded up to a multiple of the block
// size so that the NB rows of a block (j0 a multiple of NB) never wrap around
static int s2_window(const BandGeom &g, int nb, int nslot) {
    return (g.kl + g.ku + nslot * nb + nb - 1) / nb * nb;
}

template <typename C, int NB, int LC, int RC, int NSLOT>
static size_t s2_smem(const BandGeom &g) {
    return S2Layout<C, NB, LC, RC, NSLOT>::smem(s2_window(g, NB, NSLOT));
}

// the wide unit shape when it fits in shared memory
template <typename C, int NB, int LC>
static bool s2_wide(const BandGeom &g) {
    return s2_smem<C, NB, LC, 256, 2>(g) <= 227 * 1024;
}
template <typename C, int NB, int LC>
static size_t s2_smem_used(const BandGeom &g) {
    return s2_wide<C, NB, LC>(g) ? s2_smem<C, NB, LC, 256, 2>(g) : s2_smem<C, NB, LC, 128, 3>(g);
}

size_t band_solve2_smem_c64(const BandGeom &g) { return s2_smem_used<float2, NB_C64, 16>(g); }
size_t band_solve2_smem_c128(const BandGeom &g) { return s2_smem_used<double2, NB_C128, 8>(g); }
size_t band_solve2_smem_r32(const BandGeom &g) { return s2_smem_used<float, NB_C64, 16>(g); }
size_t band_solve2_smem_r64(const BandGeom &g) { return s2_smem_used<double, NB_C128, 8>(g); }

// gate = 1 if at most thr points have done == 0 (few points left: the
// narrow shape, more CTAs per point), else 0
// the shape of a refinement sweep's solve, from the number of points still
// active: the narrowest of 16, 8, 4, 2 right-hand sides per CTA whose CTAs
// for the active points fit in one wave over the SMs (a narrower shape
// shortens every block step of the chain), else the widest; gate = 0, 1, 2, 3
__global__ void solve_gate_kernel(const int32_t *__restrict__ done, int N, int L, int sms,
                                  int32_t *__restrict__ gate) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) c += done[i] == 0 ? 1 : 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        int g = 0;
        for (int k = 3; k >= 1; --k) {
            const int lc = 16 >> k;
            if ((long long)cnt * ((L + lc - 1) / lc) <= sms) { g = k; break; }
        }
        *gate = g;
    }
}

cudaError_t launch_solve_gate(const int32_t *done, int N, int L, int sms, int32_t *gate, cudaStream_t s) {
    solve_gate_kernel<<<1, 256, 0, s>>>(done, N, L, sms, gate);
    return cudaGetLastError();
}

template <typename C, int NB, int LC, int RC, int NSLOT>
static cudaError_t s2_launch(const C *ab, const int32_t *bperm, const C *dinv, C *B, const BandGeom &g,
                             int N, int n, int L, const int32_t *skip, const int32_t *gate, int want,
                             cudaStream_t s) {
    const size_t smem = s2_smem<C, NB, LC, RC, NSLOT>(g);
    const int limit = smem_optin_limit();
    if (smem > 227 * 1024 || smem > (size_t)limit) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(band_solve2_kernel<C, NB, LC, RC, NSLOT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    if (e != cudaSuccess) return e;
    dim3 grid((L + LC - 1) / LC, N);
    band_solve2_kernel<C, NB, LC, RC, NSLOT><<<grid, S2_THREADS, smem, s>>>(
        ab, bperm, dinv, B, n, g.kl, g.ku, g.ldab, L, s2_window(g, NB, NSLOT), skip, gate, want);
    return cudaGetLastError();
}

template <typename C, int NB, int LC>
static cudaError_t s2_dispatch(const C *ab, const int32_t *bperm, const C *dinv, C *B,
                               const BandGeom &g, int N, int n, int L, const int32_t *skip,
                               const int32_t *gate, int want, cudaStream_t s) {
    if (s2_wide<C, NB, LC>(g))
        return s2_launch<C, NB, LC, 256, 2>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    if constexpr (LC * 128 < S2_THREADS) {
        // two right-hand sides do not fill the 128-row units: four per CTA
        return s2_launch<C, NB, 4, 128, 3>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    } else {
        return s2_launch<C, NB, LC, 128, 3>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    }
}

cudaError_t launch_band_solve2_c64(const float2 *ab, const int32_t *bperm, const float2 *dinv,
                                   float2 *B, const BandGeom &g, int N, int n, int L,
                                   const int32_t *skip, cudaStream_t s, int lc,
                                   const int32_t *gate, int want) {
    switch (lc) {
    case 2: return s2_dispatch<float2, NB_C64, 2>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    case 4: return s2_dispatch<float2, NB_C64, 4>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    case 8: return s2_dispatch<float2, NB_C64, 8>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    default: return s2_dispatch<float2, NB_C64, 16>(ab, bperm, dinv, B, g, N, n, L, skip, gate, want, s);
    }
}
cudaError_t launch_band_solve2_r32(const float *ab, const int32_t *bperm, const float *dinv, float *B,
                                   const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s) {
    return s2_dispatch<float, NB_C64, 16>(ab, bperm, dinv, B, g, N, n, L, skip, nullptr, 0, s);
}
cudaError_t launch_band_solve2_r64(const double *ab, const int32_t *bperm, const double *dinv, double *B,
                                   const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s) {
    return s2_dispatch<double, NB_C128, 8>(ab, bperm, dinv, B, g, N, n, L, skip, nullptr, 0, s);
}
cudaError_t launch_band_solve2_c128(const double2 *ab, const int32_t *bperm, const double2 *dinv,
                                    double2 *B, const BandGeom &g, int N, int n, int L,
                                    const int32_t *skip, cudaStream_t s) {
    return s2_dispatch<double2, NB_C128, 8>(ab, bperm, dinv, B, g, N, n, L, skip, nullptr, 0, s);
}

}  // namespace rsrr
