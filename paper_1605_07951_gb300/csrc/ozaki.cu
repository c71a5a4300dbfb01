// FP64-accurate complex GEMM on the bf16 tensor cores by error-free slicing
// (the Ozaki scheme): C = alpha op(A) B + beta C with op(A) = A or A^H and
// real alpha, beta.  Used for the large products of the projection (Gram
// matrices of the sample block, Q^H R, R W, Q^H A_i Q) where native FP64
// runs at the GPU's reduced double-precision rate.
//
// 1. The complex product is one real product C~ = A~ B~ of depth K' = 2K
//    with Re/Im interleaved along K:
//      A~(i, 2k) = Re op(A)_ik,  A~(i, 2k+1) = Im op(A)_ik
//      B~(2k, j) = Re B_kj,  B~(2k+1, j) = -Im B_kj      (j < N:  Re C)
//      B~(2k, N+j) = Im B_kj,  B~(2k+1, N+j) = Re B_kj   (N + j: Im C)
// 2. Row i of A~ is scaled by 2^-e_i and column j of B~ by 2^-f_j with
//    2^(e-1) <= max |entry| < 2^e, then rounded to 55-bit fixed point
//    (exact for the largest entries, below 2^-55 absolute for the rest) and
//    split into 7 signed base-256 digits a_s in [-128, 128]:
//      x = sum_s a_s 2^(-7-8s).
//    Slice s is stored as the bf16 value a_s 2^(-8s) (exact).
// 3. Slice products of one group t = p + q are multiples of 2^(-8t) with an
//    integer part below 2^14 each; tensor-core FP32 sums of them stay exact
//    while the integer part is below 2^24.  Groups t = 0..4 get their own
//    accumulators and are folded into one int64 per output every 128 of K'
//    ((t+1) 128 2^14 <= 5 2^21 < 2^24): acc += 2^32 g_t.  Groups 5 and 6
//    (relative weight <= 2^-40) share one FP32 accumulator folded into an
//    FP32 sum; the tensor cores round such mixed-magnitude sums (measured:
//    a shared group-4..6 accumulator lost ~0.3 units of 2^-46), which at
//    this weight stays below 2^-54.  Pairs with t >= 7 (below 2^-56
//    relative) are dropped.  At most 512 folds per product keep |acc| below
//    2^62 (K is chunked beyond 32768).
// 4. C~_ij = 2^(e_i + f_j) 2^-46 (acc + 2^32 low), rounded once to FP64.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <string>

#include "rsrr.h"

#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {

constexpr int OZ_S = 7;           // slices
constexpr int OZ_BM = 64;         // CTA tile rows (M)
constexpr int OZ_BN = 64;         // CTA tile columns (of the 2N real columns)
constexpr int OZ_KC = 32;         // K' per pipeline stage
constexpr int OZ_LD = OZ_KC + 8;  // shared-memory row length (bf16): 80 bytes, conflict-free ldmatrix
constexpr int OZ_NS = 3;          // pipeline stages
constexpr int OZ_FOLD = 4;        // stages per exact fold (K' = 128)
constexpr int OZ_BCACHE = 4;      // B slices held in registers per 16-deep step
constexpr int64_t OZ_KMAX = 32768;  // complex K per chunk: <= 512 folds
constexpr int OZ_THREADS = 256;   // 8 warps: 2 (M) x 4 (N), 32 x 16 outputs each
constexpr int OZ_ROWS = OZ_S * (OZ_BM + OZ_BN);         // shared-memory rows per stage
constexpr int OZ_STAGE = OZ_ROWS * OZ_LD;                // bf16 elements per stage
constexpr size_t OZ_SMEM = sizeof(__nv_bfloat16) * OZ_STAGE * OZ_NS;  // 215040 bytes

// ----------------------------------------------------------- fixed point
// biased exponent field of |v|, subnormals and zero counted as 1
RSRR_DEV int exb_of(double v) {
    const int b = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    return b ? b : 1;
}

// round(v 2^(55 - e)) with e = E - 1022, E = largest biased exponent of the
// row; |result| <= 2^55.  Integer arithmetic only.
RSRR_DEV long long fixed55(double v, int E) {
    const long long bits = __double_as_longlong(v);
    int b = (int)((bits >> 52) & 0x7FF);
    long long mant = bits & 0xFFFFFFFFFFFFFll;
    if (b) mant |= 1ll << 52;
    else b = 1;
    const int sh = b - E + 2;  // <= 2
    long long m;
    if (sh >= 0) m = mant << sh;
    else if (sh > -62) m = (mant + (1ll << (-sh - 1))) >> (-sh);
    else m = 0;
    return bits < 0 ? -m : m;
}

// the 7 slices of a 55-bit fixed-point value as floats a_s 2^(-8s)
RSRR_DEV void digits7(long long m, float out[OZ_S]) {
#pragma unroll
    for (int s = 0; s < OZ_S - 1; ++s) {
        const int sh = 48 - 8 * s;
        const long long a = (m + (1ll << (sh - 1))) >> sh;  // round half up, |a| <= 128
        m -= a << sh;
        out[s] = (float)(int)a * ldexpf(1.f, -8 * s);
    }
    out[OZ_S - 1] = (float)(int)m * 0x1p-48f;  // remainder in [-128, 128)
}

// ----------------------------------------------------------- exponents
// E[c] = largest biased exponent in column c (contiguous, K entries); also
// written to E[c + dup] when dup > 0 (the Im-output columns of B~)
__global__ void oz_colexp_kernel(int *__restrict__ E, const double2 *__restrict__ X, int64_t ld,
                                 int K, int cols, int dup) {
    __shared__ int w[32];
    for (int c = blockIdx.x; c < cols; c += gridDim.x) {
        int m = 1;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            const double2 v = X[(int64_t)c * ld + k];
            m = max(m, max(exb_of(v.x), exb_of(v.y)));
        }
        for (int off = 16; off; off >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, off));
        if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            int r = 1;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = max(r, w[q]);
            E[c] = r;
            if (dup > 0) E[c + dup] = r;
        }
        __syncthreads();
    }
}

// E[i] = max(E[i], largest biased exponent in row i of the column-major
// rows x K matrix X); E starts at 0.  Tiles of 32 rows x 256 columns.
__global__ void oz_rowexp_kernel(int *__restrict__ E, const double2 *__restrict__ X, int64_t ld,
                                 int rows, int K) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int i = blockIdx.x * 32 + tx;
    const int k0 = blockIdx.y * 256;
    int m = 1;
    if (i < rows)
        for (int k = k0 + ty; k < min(K, k0 + 256); k += 8) {
            const double2 v = X[(int64_t)k * ld + i];
            m = max(m, max(exb_of(v.x), exb_of(v.y)));
        }
    __shared__ int w[8][32];
    w[ty][tx] = m;
    __syncthreads();
    if (ty == 0 && i < rows) {
        for (int q = 1; q < 8; ++q) m = max(m, w[q][tx]);
        atomicMax(&E[i], m);
    }
}

// ----------------------------------------------------------- slicing
// Plane layout: P[s][r][k'], row length Kp (a multiple of 32), Rp rows.
RSRR_DEV void store_slices(__nv_bfloat16 *P, size_t stride, size_t off, double re, double im, int E) {
    float dr[OZ_S], di[OZ_S];
    digits7(fixed55(re, E), dr);
    digits7(fixed55(im, E), di);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s)
        *reinterpret_cast<__nv_bfloat162 *>(P + s * stride + off) = __floats2bfloat162_rn(dr[s], di[s]);
}

RSRR_DEV void store_zero(__nv_bfloat16 *P, size_t stride, size_t off) {
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) *reinterpret_cast<__nv_bfloat162 *>(P + s * stride + off) = z;
}

// Rows built from contiguous columns of X.
//   mode 0 (A^H):  row r = conj(column r),                  r < R
//   mode 1 (B):    row r < Nc: (Re, -Im) of column r;  Nc <= r < 2Nc: (Im, Re) of column r - Nc
// Rows >= R and k >= K are written as zeros.
__global__ void oz_slice_cols_kernel(__nv_bfloat16 *__restrict__ P, const int *__restrict__ E,
                                     const double2 *__restrict__ X, int64_t ld, int mode, int R,
                                     int Nc, int K, int Rp, int Kp) {
    const size_t stride = (size_t)Rp * Kp;
    const int Kh = Kp / 2;
    for (int r = blockIdx.y; r < Rp; r += gridDim.y) {
        const int c = (mode == 1 && r >= Nc) ? r - Nc : r;
        const int Ec = (r < R) ? E[c] : 1;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Kh; k += gridDim.x * blockDim.x) {
            const size_t off = (size_t)r * Kp + 2 * (size_t)k;
            if (r >= R || k >= K) {
                store_zero(P, stride, off);
                continue;
            }
            const double2 v = X[(int64_t)c * ld + k];
            double re = v.x, im = -v.y;
            if (mode == 1 && r >= Nc) { re = v.y; im = v.x; }
            store_slices(P, stride, off, re, im, Ec);
        }
    }
}

// Rows of A itself (column-major M x K, row i strided): 32 x 32 tiles
// transposed through shared memory.  Rows >= M and k >= K are zeros.
__global__ void oz_slice_rows_kernel(__nv_bfloat16 *__restrict__ P, const int *__restrict__ E,
                                     const double2 *__restrict__ A, int64_t lda, int M, int K, int Mp,
                                     int Kp) {
    __shared__ double2 t[32][33];
    const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + tx, k = k0 + r;
        t[r][tx] = (i < M && k < K) ? A[(int64_t)k * lda + i] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const size_t stride = (size_t)Mp * Kp;
    const int Kh = Kp / 2;
    for (int r = ty; r < 32; r += 8) {
        const int i = i0 + r, k = k0 + tx;
        if (i >= Mp || k >= Kh) continue;
        const size_t off = (size_t)i * Kp + 2 * (size_t)k;
        if (i >= M || k >= K) {
            store_zero(P, stride, off);
            continue;
        }
        const double2 v = t[tx][r];
        store_slices(P, stride, off, v.x, v.y, E[i]);
    }
}

// Stage images for the tensor-core kernel: the slices of one operand tile
// (TR rows, 16 of K') stored in exactly the order that kernel keeps them in
// shared memory, so that one bulk copy moves one operand of a stage.
//   chunk (rb, ks): rows TR rb .. +TR-1, K' 16 ks .. +15; OZ_S TR 16 elements
//   element (s, row, k') of a chunk at  s ss + kc kcs + 8 (row % TR) + k' % 8,
//   kc = (k' % 16) / 8 the core-matrix column (8 rows x 16 bytes a core matrix)
//   per-slice operand (A):          ss = 16 TR,  kcs = 8 TR
//   slices stacked per core column (B, read as one N = 64 q operand):
//                                   ss = 8 TR,   kcs = 8 OZ_S TR
// Rows as in oz_slice_cols_kernel (mode 0, 1) or rows of the column-major X
// itself (mode 2, as oz_slice_rows_kernel); rows >= R and k >= K are zeros.
// One warp per 8 rows x 4 complex K (a core matrix of every slice): lane =
// 4 (row % 8) + k % 4, so every slice store of a warp is 128 contiguous bytes.
__global__ void oz_slice_tiled_kernel(__nv_bfloat16 *__restrict__ P, const int *__restrict__ E,
                                      const double2 *__restrict__ X, int64_t ld, int mode, int R,
                                      int Nc, int K, int Rp, int Kp, int TR, int stacked) {
    const int lane = threadIdx.x & 31;
    const int64_t nrg = Rp / 8, nkg = Kp / 8, total = nrg * nkg;
    const int64_t nks = Kp / 16;
    const size_t ss = stacked ? 8 * (size_t)TR : 16 * (size_t)TR;
    const size_t kcs = stacked ? 8 * (size_t)OZ_S * TR : 8 * (size_t)TR;
    const size_t chunk = (size_t)OZ_S * TR * 16;
    const int64_t wstep = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += wstep) {
        // consecutive warps along the contiguous direction of X
        const int64_t rg = mode == 2 ? w % nrg : w / nkg;
        const int64_t kg = mode == 2 ? w / nrg : w % nkg;
        const int r = (int)(8 * rg) + (lane >> 2);
        const int k = (int)(4 * kg) + (lane & 3);  // complex index, k' = 2k
        const size_t off = ((size_t)(r / TR) * nks + (size_t)(kg >> 1)) * chunk + (size_t)(kg & 1) * kcs +
                           8 * (size_t)(r % TR) + 2 * (lane & 3);
        if (r >= R || k >= K) {
            store_zero(P, ss, off);
            continue;
        }
        if (mode == 2) {
            const double2 v = X[(int64_t)k * ld + r];
            store_slices(P, ss, off, v.x, v.y, E[r]);
        } else {
            const int c = (mode == 1 && r >= Nc) ? r - Nc : r;
            const double2 v = X[(int64_t)c * ld + k];
            double re = v.x, im = -v.y;
            if (mode == 1 && r >= Nc) { re = v.y; im = v.x; }
            store_slices(P, ss, off, re, im, E[c]);
        }
    }
}

// ----------------------------------------------------------- the GEMM
RSRR_DEV void cp_async16(unsigned saddr, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem));
}
RSRR_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
RSRR_DEV void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

RSRR_DEV void ldmatrix_x4(unsigned r[4], unsigned saddr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr));
}

RSRR_DEV void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// round(f 2^32) for a group sum f of groups t <= 4, in integer instructions.
// Such an f is an integer multiple of 2^-32 below 2^24 in magnitude (step 3
// above), so f = m 2^(e-150) with a 24-bit m and e >= 95, and f 2^32 =
// m 2^(e-118) is an integer below 2^56: the shift loses only zero bits and
// the result is exactly the float-to-int64 conversion of f 2^32, without the
// conversion unit (it shares the GPU's slow double-precision pipe).
RSRR_DEV long long scaled_group_to_ll(float f) {
    const int bits = __float_as_int(f);
    const int e = (bits >> 23) & 0xFF;
    if (e == 0) return 0;  // +-0 (subnormals cannot occur: |f| >= 2^-32)
    long long m = (long long)((bits & 0x7FFFFF) | 0x800000);
    const int sh = e - 118;
    m = sh >= 0 ? (m << sh) : (m >> -sh);
    return bits < 0 ? -m : m;
}

// One CTA: a 64 x 64 tile of C~ over K' range [sp kchunk, (sp+1) kchunk).
// W != null: FP64 partial tile into W[sp][i][j'] (Mp x Np, row major).
// W == null: C = alpha C~ + beta C written directly (one split).
// upper_only: tiles strictly below the block diagonal of each half skip.
__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __nv_bfloat16 *__restrict__ As, const __nv_bfloat16 *__restrict__ Bs,
               const int *__restrict__ Ea, const int *__restrict__ Eb, double *__restrict__ W,
               double2 *__restrict__ C, int64_t ldc, int M, int N, int Mp, int Np, int Kp, int kchunk,
               int halfN_tiles, int upper_only, double alpha, double beta) {
    const int bm = blockIdx.x, bn = blockIdx.y, sp = blockIdx.z;
    if (upper_only && bm > (bn % halfN_tiles)) return;
    extern __shared__ __align__(128) unsigned char oz_smem[];
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(oz_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int g = lane >> 2, tq = lane & 3;
    const int m0 = bm * OZ_BM, n0 = bn * OZ_BN;
    const int kbeg = sp * kchunk;
    const int kend = min(Kp, kbeg + kchunk);
    const int nk = kend > kbeg ? (kend - kbeg) / OZ_KC : 0;
    const size_t sA = (size_t)Mp * Kp, sB = (size_t)Np * Kp;

    float gs[6][2][2][4];
    long long acc[2][2][4];
    float low[2][2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc[a][b][q] = 0;
                low[a][b][q] = 0.f;
#pragma unroll
                for (int t = 0; t < 6; ++t) gs[t][a][b][q] = 0.f;
            }

    // stage rows: slice s, rows 0..63 from A~, 64..127 from B~
    auto load_stage = [&](int slot, int k0) {
        const unsigned dst = sbase + (unsigned)(slot * OZ_STAGE * 2);
        for (int q = tid; q < OZ_ROWS * 4; q += OZ_THREADS) {
            const int row = q >> 2, c = q & 3;
            const int s = row >> 7, rr = row & 127;
            const __nv_bfloat16 *src =
                (rr < OZ_BM) ? As + s * sA + (size_t)(m0 + rr) * Kp + k0 + c * 8
                             : Bs + s * sB + (size_t)(n0 + rr - OZ_BM) * Kp + k0 + c * 8;
            cp_async16(dst + (unsigned)((row * OZ_LD + c * 8) * 2), src);
        }
    };

#pragma unroll
    for (int st = 0; st < OZ_NS - 1; ++st) {
        if (st < nk) load_stage(st, kbeg + st * OZ_KC);
        cp_async_commit();
    }
    // per-lane ldmatrix row offsets (bf16 elements within one slice)
    const int li = lane & 7, mi = lane >> 3;
    const int a_off = (wm * 32 + (mi & 1) * 8 + li) * OZ_LD + (mi >> 1) * 8;
    const int b_off = (OZ_BM + wn * 16 + (mi >> 1) * 8 + li) * OZ_LD + (mi & 1) * 8;

    for (int it = 0; it < nk; ++it) {
        cp_async_wait<OZ_NS - 2>();
        __syncthreads();
        {
            const int nx = it + OZ_NS - 1;
            if (nx < nk) load_stage(nx % OZ_NS, kbeg + nx * OZ_KC);
            cp_async_commit();
        }
        const unsigned st = sbase + (unsigned)((it % OZ_NS) * OZ_STAGE * 2);
#pragma unroll
        for (int kk = 0; kk < OZ_KC; kk += 16) {
            // B slices 0..3 stay in registers for the whole step; 4..6 (used
            // by p <= 2 only) are loaded where needed
            unsigned bfr[OZ_BCACHE][4];
#pragma unroll
            for (int q = 0; q < OZ_BCACHE; ++q)
                ldmatrix_x4(bfr[q], st + (unsigned)((q * (OZ_BM + OZ_BN) * OZ_LD + b_off + kk) * 2));
#pragma unroll
            for (int p = 0; p < OZ_S; ++p) {
                unsigned afr[2][4];
                const unsigned pa = st + (unsigned)((p * (OZ_BM + OZ_BN) * OZ_LD + a_off + kk) * 2);
                ldmatrix_x4(afr[0], pa);
                ldmatrix_x4(afr[1], pa + 16 * OZ_LD * 2);
#pragma unroll
                for (int q = 0; q < OZ_S - p; ++q) {
                    const int t = p + q < 5 ? p + q : 5;
                    unsigned bx[4];
                    if (q < OZ_BCACHE) {
#pragma unroll
                        for (int r = 0; r < 4; ++r) bx[r] = bfr[q < OZ_BCACHE ? q : 0][r];
                    } else {
                        ldmatrix_x4(bx, st + (unsigned)((q * (OZ_BM + OZ_BN) * OZ_LD + b_off + kk) * 2));
                    }
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 2; ++b) mma_bf16(gs[t][a][b], afr[a], bx[2 * b], bx[2 * b + 1]);
                }
            }
        }
        if ((it + 1) % OZ_FOLD == 0 || it == nk - 1) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
#pragma unroll
                        for (int t = 0; t < 5; ++t) {
                            acc[a][b][q] += scaled_group_to_ll(gs[t][a][b][q]);
                            gs[t][a][b][q] = 0.f;
                        }
                        low[a][b][q] += gs[5][a][b][q];
                        gs[5][a][b][q] = 0.f;
                    }
        }
    }
    cp_async_wait<0>();

#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = m0 + wm * 32 + a * 16 + g + (q >= 2 ? 8 : 0);
                const int jj = n0 + wn * 16 + b * 8 + 2 * tq + (q & 1);
                const double v = ldexp((double)acc[a][b][q] + (double)low[a][b][q] * 0x1p32,
                                       Ea[i] + Eb[jj] - 2090);
                if (W) {
                    W[(size_t)sp * Mp * Np + (size_t)i * Np + jj] = v;
                } else if (i < M && jj < 2 * N) {
                    const int part = jj >= N, j = jj - part * N;
                    double *c = reinterpret_cast<double *>(C + (int64_t)j * ldc + i) + part;
                    double r = alpha * v;
                    if (beta != 0.0) r = fma(beta, *c, r);
                    *c = r;
                }
            }
}

// ----------------------------------------------------------- tcgen05 path
// The same products on the 5th-generation tensor cores: a CTA of 256 threads
// owns a 128 x 64 tile of C~.  Per 16-deep stage of K' the 7 A slices (128
// rows) and the 7 B slices (64 rows each, stacked to 448 rows) arrive by two
// bulk copies of the TMA engine (the stage images of oz_slice_tiled_kernel,
// 28 and 14 KB, contiguous in global memory; issued by one thread, completion
// counted in bytes on the stage's mbarrier) in the K-major core-matrix layout
// (8 rows x 16 bytes per core matrix, no swizzle), in a ring of OZT_NST
// stages; a slot is refilled once the MMAs that read it have committed.  One thread issues
// 10 tcgen05.mma per stage (M = 128, N = 64..256, bf16 -> FP32 in tensor
// memory): every group t = p + q has its own 64-column region of tensor
// memory (7 regions, 448 of the 512 columns), so the pairs of one A slice
// (q = 0 .. 6 - p) are MMAs over consecutive B slices into consecutive
// regions, four slices (N = 256) at a time; the issuing thread never waits
// at a CTA-wide barrier except for the folds.  Groups t <= 4 hold at most
// (t+1) 2^14 per K' element, so every 192 of K' (and at the end) all threads
// wait for the MMAs (tcgen05.commit -> mbarrier), read their part of the
// regions (tcgen05.ld; warp w of 16 reads TMEM lanes 32 (w % 4) .. +31 = tile
// rows, columns 16 (w / 4) .. +15), fold groups 0..4 into 64-bit integers and add
// groups 5..6 (relative weight <= 2^-40, rounded by design) into an FP32 sum;
// the next MMAs restart every region.  Every mbarrier wait is bounded; a wait that runs out is
// counted in the caller's device status word, and from then on the CTA issues no further TMA copy
// or MMA (the copy and MMA threads share an abort flag in shared memory; skipped stages still
// commit their mbarriers so that the folds stay balanced), waits (bounded) for the copies it did
// issue, and finishes without hanging.
constexpr int OZT_BM = 128;
constexpr int OZT_BN = 64;
constexpr int OZT_KC = 16;
constexpr int OZT_THREADS = 512;                 // 16 warps: 4 lane quarters x 4 column groups
constexpr int OZT_CPT = OZT_BN / (OZT_THREADS / 128);  // tile columns a thread folds (16)
constexpr int OZT_PRODUCER = OZT_THREADS / 2;    // the copy thread (first lane of the upper half)
constexpr int OZT_A_SLICE = OZT_BM * OZT_KC * 2;           // bytes of one A slice per stage
constexpr int OZT_B_SLICE = OZT_BN * OZT_KC * 2;           // bytes of one B slice per stage
constexpr int OZT_STAGE = OZ_S * (OZT_A_SLICE + OZT_B_SLICE);
constexpr int OZT_NST = 5;
constexpr int OZT_DIST = OZT_NST - 2;  // stages the copies run ahead of a fold
// after the stages: 2 NST + 1 mbarriers, the TMEM address, the abort flag
constexpr int OZT_TSLOT = 16 * OZT_NST + 16;
constexpr int OZT_ABORT = OZT_TSLOT + 16;
constexpr size_t OZT_SMEM = (size_t)OZT_NST * OZT_STAGE + 128;
static_assert(OZT_ABORT + 4 <= 128, "barrier area");
static_assert(OZT_SMEM <= 232448, "shared memory per CTA");
// stage layout, K-major core matrices (8 rows x 16 bytes), no swizzle: per
// K-column of core matrices (8 of K) all rows of an operand are contiguous,
// 16 bytes a row, so one TMA box of 16 bytes x rows fills one such column
constexpr uint32_t OZT_SBO = 128;                          // next 8-row group
constexpr uint32_t OZT_LBO_A = OZT_BM * 16;                // next core column of an A slice
constexpr uint32_t OZT_LBO_B = OZ_S * OZT_BN * 16;         // next core column of the stacked B
constexpr int OZT_FOLD = 12;                      // stages per exact fold (K' = 192)
constexpr long long OZT_WAIT_LIMIT = 1LL << 22;
static_assert((4 + 1) * OZT_FOLD * OZT_KC * 16384 < (1 << 24), "group sums must stay exact in FP32");
static_assert(OZ_S * OZT_BN <= 512, "one tensor-memory region per group");

// shared-memory matrix descriptor: K-major, no swizzle, start / LBO (next core
// matrix along K) / SBO (next 8-row group) in 16-byte units, version 1
RSRR_DEV uint64_t umma_desc(uint32_t saddr, uint32_t lbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((OZT_SBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = n
RSRR_DEV uint32_t umma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZT_BM >> 4) << 24);
}
RSRR_DEV void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
RSRR_DEV void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(mbar) : "memory");
}
// bulk copy (TMA engine) of `bytes` contiguous bytes into shared memory,
// completion counted in bytes on mbar; both addresses 16-byte aligned, bytes
// a multiple of 16
RSRR_DEV void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
RSRR_DEV void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
RSRR_DEV bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = OZT_WAIT_LIMIT) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
// bounded wait that also gives up as soon as another thread of the CTA has
// raised the abort flag (the copy and MMA threads; folds and the final drain
// use the plain bounded wait so that operations in flight still land)
RSRR_DEV bool mbar_wait_or_abort(uint32_t mbar, uint32_t parity, volatile int *abort_flag,
                                 long long limit = OZT_WAIT_LIMIT) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        if (*abort_flag) return false;
    }
    return false;
}
RSRR_DEV void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// The integer n of a group sum g = n 2^(-8t) with |n| < 2^24 (t <= 4; the
// fold cadence bounds n), exactly, in FP32 and integer ALU operations (the
// conversion instructions are slow on this GPU).  s = 2^(8t), s12 = 2^(8t-12):
//   r  = fma(g, s12, 1.5 2^23) = 1.5 2^23 + h with h = rint(n 2^-12), |h| <= 2^12:
//        the sum lies in [2^23, 2^24), where floats are the integers
//   lo = n - 2^12 h (|lo| <= 2^11), an exact FMA;  r2 = 1.5 2^23 + lo, exact
//   bits(r) = 0x4B400000 + h and bits(r2) = 0x4B400000 + lo, so
//   n = 2^12 bits(r) + bits(r2) - 4097 0x4B400000  (mod 2^32; |n| < 2^31)
RSRR_DEV int group_int(float g, float s12, float s) {
    const float M = 12582912.f;  // 1.5 2^23
    const float r = fmaf(g, s12, M);
    const float lo = fmaf(r - M, -4096.f, g * s);
    const float r2 = lo + M;
    return (int)(((uint32_t)__float_as_int(r) << 12) + (uint32_t)__float_as_int(r2) - 4097u * 0x4B400000u);
}

__global__ void __launch_bounds__(OZT_THREADS, 1)
oz_gemm_tc_kernel(const __nv_bfloat16 *__restrict__ As, const __nv_bfloat16 *__restrict__ Bs,
                  const int *__restrict__ Ea, const int *__restrict__ Eb, double *__restrict__ W,
                  double2 *__restrict__ C, int64_t ldc, int M, int N, int Mp, int Np, int Kp, int kchunk,
                  int halfN_tiles, int upper_only, double alpha, double beta,
                  unsigned int *__restrict__ status) {
    const int bm = blockIdx.x, bn = blockIdx.y, sp = blockIdx.z;
    if (upper_only && OZT_BM * bm > OZT_BN * (bn % halfN_tiles) + OZT_BN - 1) return;
    extern __shared__ __align__(1024) unsigned char ozt_smem[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(ozt_smem);
    const uint32_t mb_full = sbase + OZT_NST * OZT_STAGE;  // OZT_NST: stage's bytes landed (TMA)
    const uint32_t mb_empty = mb_full + 8 * OZT_NST;       // OZT_NST: stage's MMAs done
    const uint32_t mb_fold = mb_empty + 8 * OZT_NST;       // all MMAs so far done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(ozt_smem + OZT_NST * OZT_STAGE + OZT_TSLOT);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(ozt_smem + OZT_NST * OZT_STAGE + OZT_ABORT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = bm * OZT_BM, n0 = bn * OZT_BN;
    const int kbeg = sp * kchunk;
    const int kend = min(Kp, kbeg + kchunk);
    const int nk = kend > kbeg ? (kend - kbeg) / OZT_KC : 0;
    // roles: thread OZT_PRODUCER copies the stages, thread 0 issues the MMAs,
    // all sixteen warps fold (warp w: TMEM lanes 32 (w % 4) .., columns
    // 16 (w / 4) ..)
    const bool producer = tid >= OZT_PRODUCER;

    if (tid == 0) {
        for (int q = 0; q < OZT_NST; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_full + 8 * q));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_empty + 8 * q));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb_fold));
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    const int lrow = 32 * (warp & 3) + lane, lcol = OZT_CPT * (warp >> 2);
    const uint32_t tpart = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)lcol;

    long long acc[OZT_CPT];
    float low[OZT_CPT];
#pragma unroll
    for (int c = 0; c < OZT_CPT; ++c) {
        acc[c] = 0;
        low[c] = 0.f;
    }
    bool ok = true;
    int folds = 0;
    auto is_fold = [&](int st) { return ((st + 1) % OZT_FOLD) == 0 || st == nk - 1; };
    // every warp, after the MMAs of a fold stage: regions 0..4 into the integers
    auto fold_part = [&]() {
        if (!mbar_wait(mb_fold, folds & 1)) {
            ok = false;
            *abort_flag = 1;
        }
        ++folds;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        static_assert(OZT_CPT == 16, "one 16-column TMEM load per region");
#pragma unroll
        for (int t = 0; t < OZ_S; ++t) {
            uint32_t r[16];
            tmem_ld16(tpart + (uint32_t)(t * OZT_BN), r);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (t < 5)
                    acc[j] += (long long)group_int(__uint_as_float(r[j]), 0x1p-12f * (float)(1ull << (8 * t)),
                                                   (float)(1ull << (8 * t)))
                              << (32 - 8 * t);
                else
                    low[j] += __uint_as_float(r[j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        asm volatile("bar.sync 1, %0;\n" ::"n"(OZT_THREADS) : "memory");  // regions free again
    };
    if (producer) {
        // one thread issues the stage copies (one stage image of each operand),
        // OZT_DIST stages ahead of the fold that follows a stage
        const size_t nks = (size_t)(Kp / OZT_KC);
        const __nv_bfloat16 *srcA = As + (size_t)bm * nks * (OZ_S * OZT_BM * OZT_KC);
        const __nv_bfloat16 *srcB = Bs + (size_t)bn * nks * (OZ_S * OZT_BN * OZT_KC);
        int issued = 0;  // stages whose copies were issued (all of them unless a wait ran out)
        for (int st = 0; st < nk + OZT_DIST; ++st) {
            if (st < nk && tid == OZT_PRODUCER && !*abort_flag) {
                const int slot = st % OZT_NST;
                // slot st % NST was last read by the MMAs of stage st - NST
                if (st >= OZT_NST &&
                    !mbar_wait_or_abort(mb_empty + 8 * slot, ((st / OZT_NST) - 1) & 1, abort_flag)) {
                    ok = false;
                    *abort_flag = 1;
                }
            }
            if (st < nk && tid == OZT_PRODUCER && !*abort_flag) {
                const int slot = st % OZT_NST;
                const uint32_t full = mb_full + 8 * slot;
                mbar_expect_tx(full, (uint32_t)OZT_STAGE);
                const uint32_t a0 = sbase + (uint32_t)(slot * OZT_STAGE);
                const uint32_t b0 = a0 + OZ_S * OZT_A_SLICE;
                const size_t ks = (size_t)(kbeg / OZT_KC + st);
                bulk_load(a0, srcA + ks * (OZ_S * OZT_BM * OZT_KC), (uint32_t)(OZ_S * OZT_A_SLICE), full);
                bulk_load(b0, srcB + ks * (OZ_S * OZT_BN * OZT_KC), (uint32_t)(OZ_S * OZT_B_SLICE), full);
                issued = st + 1;
            }
            __syncwarp();
            const int done = st - OZT_DIST;
            if (done >= 0 && is_fold(done)) fold_part();
        }
        // every copy that was issued has landed before the CTA leaves (waits
        // bounded; the last issued stage of each slot is its latest phase)
        if (tid == OZT_PRODUCER)
            for (int st = max(0, issued - OZT_NST); st < issued; ++st)
                ok = mbar_wait(mb_full + 8 * (st % OZT_NST), (st / OZT_NST) & 1) && ok;
        __syncwarp();
    } else {
        for (int it = 0; it < nk; ++it) {
            if (tid == 0) {
                const int slot = it % OZT_NST;
                bool go = !*abort_flag;
                if (go && !mbar_wait_or_abort(mb_full + 8 * slot, (it / OZT_NST) & 1, abort_flag)) {
                    ok = false;
                    *abort_flag = 1;
                    go = false;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = sbase + (uint32_t)(slot * OZT_STAGE);
                const uint32_t b0 = a0 + OZ_S * OZT_A_SLICE;
                const uint32_t keep = (it % OZT_FOLD) == 0 ? 0u : 1u;  // all regions restart after a fold
#pragma unroll
                for (int p = 0; p < OZ_S; ++p) {
                    if (!go) break;  // no MMA on a stage whose copies did not land
                    const uint64_t ad = umma_desc(a0 + p * OZT_A_SLICE, OZT_LBO_A);
                    // groups p .. 6 (q = 0 .. 6 - p): consecutive B slices into
                    // consecutive regions, at most 4 slices (N = 256) per MMA
#pragma unroll
                    for (int q0 = 0; q0 <= OZ_S - 1 - p; q0 += 4) {
                        const int nq = min(4, OZ_S - p - q0);
                        umma_bf16(tmem + (uint32_t)((p + q0) * OZT_BN), ad, umma_desc(b0 + q0 * OZT_BN * 16, OZT_LBO_B),
                                  umma_idesc(nq * OZT_BN), p == 0 ? keep : 1u);
                    }
                }
                // committed whether or not MMAs were issued: the slot and the
                // fold barrier complete once every earlier MMA has finished
                umma_commit(mb_empty + 8 * slot);
                if (is_fold(it)) umma_commit(mb_fold);
            }
            __syncwarp();
            if (is_fold(it)) fold_part();
        }
    }
    if (!ok && lane == 0) atomicAdd(status, 1u);

    const int i = m0 + lrow;
    const int ea = Ea[i];
#pragma unroll
    for (int c = 0; c < OZT_CPT; ++c) {
        const int jj = n0 + lcol + c;
        const double v = ldexp((double)acc[c] + (double)low[c] * 0x1p32, ea + Eb[jj] - 2090);
        if (W) {
            W[(size_t)sp * Mp * Np + (size_t)i * Np + jj] = v;
        } else if (i < M && jj < 2 * N) {
            const int part = jj >= N, j = jj - part * N;
            double *cp = reinterpret_cast<double *>(C + (int64_t)j * ldc + i) + part;
            double r = alpha * v;
            if (beta != 0.0) r = fma(beta, *cp, r);
            *cp = r;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
}

// Failure-detection check of the bounded wait: one thread waits on an
// mbarrier that nothing arrives on; the wait gives up after `limit` tries and
// is counted in the status word, exactly as in the tensor-core kernel.
__global__ void ozt_wait_check_kernel(long long limit, unsigned int *status) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    if (!mbar_wait(a, 0, limit)) atomicAdd(status, 1u);
}

cudaError_t launch_wait_check(long long limit, unsigned int *status, cudaStream_t s) {
    ozt_wait_check_kernel<<<1, 32, 0, s>>>(limit, status);
    return cudaGetLastError();
}

// C = alpha sum_s W[s] + beta C (fixed order over the splits)
__global__ void oz_combine_kernel(double2 *__restrict__ C, int64_t ldc, const double *__restrict__ W,
                                  int M, int N, int Mp, int Np, int splits, double alpha, double beta,
                                  int upper_only, int bm) {
    const int64_t total = (int64_t)M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % M), j = (int)(q / M);
        if (upper_only && bm * (i / bm) > OZ_BN * (j / OZ_BN) + OZ_BN - 1) continue;
        double re = 0.0, im = 0.0;
        for (int s = 0; s < splits; ++s) {
            const double *Wp = W + (size_t)s * Mp * Np + (size_t)i * Np;
            re += Wp[j];
            im += Wp[N + j];
        }
        double2 r = make_double2(alpha * re, alpha * im);
        if (beta != 0.0) {
            const double2 c = C[(int64_t)j * ldc + i];
            r.x = fma(beta, c.x, r.x);
            r.y = fma(beta, c.y, r.y);
        }
        C[(int64_t)j * ldc + i] = r;
    }
}

__global__ void oz_mirror_kernel(double2 *__restrict__ C, int64_t ldc, int n) {
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        if (i > j) {
            const double2 v = C[(int64_t)i * ldc + j];
            C[(int64_t)j * ldc + i] = make_double2(v.x, -v.y);
        } else if (i == j) {
            C[(int64_t)j * ldc + i].y = 0.0;  // the rounded low groups leave ~2^-56 here
        }
    }
}

// C = beta C (K = 0 or alpha = 0)
__global__ void oz_scale_kernel(double2 *__restrict__ C, int64_t ldc, int M, int N, double beta) {
    const int64_t total = (int64_t)M * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % M), j = (int)(q / M);
        double2 &c = C[(int64_t)j * ldc + i];
        c = beta == 0.0 ? make_double2(0.0, 0.0) : make_double2(beta * c.x, beta * c.y);
    }
}

// ----------------------------------------------------------- host side
static int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
static int grid_for(int64_t work) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 8));
}

namespace {
struct OzPlan {
    int64_t Mp, Np, Kc, Kp;  // Kc: complex K per chunk
    int splits;
    int64_t kchunk;          // K' per split
    size_t bytes;
};

size_t plan_bytes(int64_t Mp, int64_t Np, int64_t Kp, int splits) {
    size_t b = rup((int64_t)sizeof(__nv_bfloat16) * OZ_S * Mp * Kp, 256);
    b += rup((int64_t)sizeof(__nv_bfloat16) * OZ_S * Np * Kp, 256);
    b += rup((int64_t)sizeof(int) * (Mp + Np), 256);
    if (splits > 1) b += rup((int64_t)sizeof(double) * splits * Mp * Np, 256);
    return b;
}

// splits of K that balance the waves over the 152 SMs (one CTA per SM)
int choose_splits(int64_t tiles, int64_t Kp) {
    int best = 1;
    double best_cost = 1e300;
    for (int s = 1; s <= 32; ++s) {
        if (s > 1 && Kp / s < (int64_t)OZ_FOLD * OZ_KC * 2) break;
        const double waves = (double)((tiles * s + 151) / 152);
        const double cost = waves / s * (1.0 + 0.01 * s);
        if (cost < best_cost - 1e-12) {
            best_cost = cost;
            best = s;
        }
    }
    return best;
}

// computed tiles of a bm x 64 tiling (upper block triangle only for Hermitian results)
int64_t tile_count(int64_t Mp, int64_t Np, int bm, bool upper, int64_t halfN) {
    if (!upper) return (Mp / bm) * (Np / OZ_BN);
    int64_t t = 0;
    for (int64_t a = 0; a < Mp / bm; ++a)
        for (int64_t b = 0; b < Np / OZ_BN; ++b)
            if (bm * a <= OZ_BN * (b % halfN) + OZ_BN - 1) ++t;
    return t;
}

OzPlan make_plan(int M, int N, int K, bool hermitian, size_t ws_bytes, int bm) {
    OzPlan p{};
    p.Mp = rup(M, bm);
    p.Np = rup(2 * (int64_t)N, OZ_BN);
    const int64_t tiles = (p.Mp / bm) * (p.Np / OZ_BN) / (hermitian ? 2 : 1);
    const int64_t Kall = std::max(K, 1);
    auto fit = [&](int64_t kc) {
        p.Kc = kc;
        p.Kp = rup(2 * p.Kc, OZ_KC);
        p.splits = choose_splits(std::max<int64_t>(tiles, 1), p.Kp);
        while (p.splits > 1 && plan_bytes(p.Mp, p.Np, p.Kp, p.splits) > ws_bytes) --p.splits;
        p.bytes = plan_bytes(p.Mp, p.Np, p.Kp, p.splits);
        return p.bytes <= ws_bytes;
    };
    int64_t kc = std::min<int64_t>(Kall, OZ_KMAX);
    while (!fit(kc) && kc > 16) kc = std::max<int64_t>(16, rup(kc / 2, 16));  // chunk K to fit
    // chunks of equal depth
    const int64_t nch = (Kall + kc - 1) / kc;
    if (nch > 1) fit(std::min(kc, rup((Kall + nch - 1) / nch, 16)));
    p.kchunk = rup((p.Kp + p.splits - 1) / p.splits, OZ_KC);
    p.splits = (int)((p.Kp + p.kchunk - 1) / p.kchunk);
    return p;
}
}  // namespace

size_t ozaki_workspace_bytes(int M, int N, int K, bool hermitian) {
    return std::max(make_plan(M, N, K, hermitian, SIZE_MAX, OZ_BM).bytes,
                    make_plan(M, N, K, hermitian, SIZE_MAX, OZT_BM).bytes);
}

double ozaki_tc_flops(int M, int N, int K, bool hermitian, bool legacy) {
    if (M <= 0 || N <= 0 || K <= 0) return 0.0;
    const int bm = legacy ? OZ_BM : OZT_BM;
    const OzPlan p = make_plan(M, N, K, hermitian, SIZE_MAX, bm);
    const double pairs = OZ_S * (OZ_S + 1) / 2;
    const bool upper = hermitian && M == N && (N % OZ_BN) == 0;
    const double tiles = (double)tile_count(p.Mp, p.Np, bm, upper, upper ? N / OZ_BN : p.Np / OZ_BN);
    return 2.0 * pairs * tiles * bm * OZ_BN * (double)p.Kp;
}

cudaError_t ozaki_zgemm(int M, int N, int K, bool conjA, const double2 *A, int64_t lda,
                        const double2 *B, int64_t ldb, double2 *C, int64_t ldc, double alpha,
                        double beta, bool hermitian, void *ws, size_t ws_bytes, cudaStream_t s,
                        int64_t *launches, EventPool *timer, double *tc_flops, bool legacy,
                        unsigned int *status) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!legacy && !status) return cudaErrorInvalidValue;
    cudaError_t e;
    if (K <= 0 || alpha == 0.0) {
        oz_scale_kernel<<<grid_for((int64_t)M * N), 256, 0, s>>>(C, ldc, M, N, beta);
        if (launches) *launches += 1;
        return cudaGetLastError();
    }
    if (hermitian && (M != N || !conjA || A != B || lda != ldb)) hermitian = false;
    const int bm = legacy ? OZ_BM : OZT_BM;
    const OzPlan p = make_plan(M, N, K, hermitian, ws_bytes, bm);
    if (p.bytes > ws_bytes) return cudaErrorMemoryAllocation;
    if (legacy)
        e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
    else
        e = cudaFuncSetAttribute(oz_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZT_SMEM);
    if (e != cudaSuccess) return e;
    char *w = static_cast<char *>(ws);
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(w);
    w += rup((int64_t)sizeof(__nv_bfloat16) * OZ_S * p.Mp * p.Kp, 256);
    __nv_bfloat16 *Bs = reinterpret_cast<__nv_bfloat16 *>(w);
    w += rup((int64_t)sizeof(__nv_bfloat16) * OZ_S * p.Np * p.Kp, 256);
    int *Ea = reinterpret_cast<int *>(w);
    int *Eb = Ea + p.Mp;
    w += rup((int64_t)sizeof(int) * (p.Mp + p.Np), 256);
    double *Wp = p.splits > 1 ? reinterpret_cast<double *>(w) : nullptr;
    const bool upper = hermitian && (N % OZ_BN) == 0;
    const int halfN_tiles = upper ? N / OZ_BN : (int)(p.Np / OZ_BN);

    for (int64_t kc0 = 0; kc0 < K; kc0 += p.Kc) {
        const int Kc = (int)std::min<int64_t>(p.Kc, K - kc0);
        const double b = kc0 == 0 ? beta : 1.0;
        const double2 *Ak = conjA ? A + kc0 : A + kc0 * lda;
        const double2 *Bk = B + kc0;
        if ((e = cudaMemsetAsync(Ea, 0, sizeof(int) * (p.Mp + p.Np), s)) != cudaSuccess) return e;
        if (conjA)
            oz_colexp_kernel<<<std::min(M, 65535), 256, 0, s>>>(Ea, Ak, lda, Kc, M, 0);
        else
            oz_rowexp_kernel<<<dim3((unsigned)((M + 31) / 32), (unsigned)((Kc + 255) / 256)), 256, 0, s>>>(
                Ea, Ak, lda, M, Kc);
        oz_colexp_kernel<<<std::min(N, 65535), 256, 0, s>>>(Eb, Bk, ldb, Kc, N, N);
        if (legacy) {
            const int kx = (int)std::min<int64_t>((p.Kp / 2 + 255) / 256, 64);
            if (conjA)
                oz_slice_cols_kernel<<<dim3(kx, (unsigned)std::min<int64_t>(p.Mp, 65535)), 256, 0, s>>>(
                    As, Ea, Ak, lda, 0, M, M, Kc, (int)p.Mp, (int)p.Kp);
            else
                oz_slice_rows_kernel<<<dim3((unsigned)(p.Mp / 32), (unsigned)((p.Kp / 2 + 31) / 32)), 256, 0,
                                       s>>>(As, Ea, Ak, lda, M, Kc, (int)p.Mp, (int)p.Kp);
            oz_slice_cols_kernel<<<dim3(kx, (unsigned)std::min<int64_t>(p.Np, 65535)), 256, 0, s>>>(
                Bs, Eb, Bk, ldb, 1, 2 * N, N, Kc, (int)p.Np, (int)p.Kp);
        } else {
            // stage images: one warp per 8 rows x 8 of K'
            auto blocks = [](int64_t rows, int64_t kp) {
                return (unsigned)std::max<int64_t>(1, std::min<int64_t>(rows / 8 * (kp / 8) / 8, 152 * 16));
            };
            oz_slice_tiled_kernel<<<blocks(p.Mp, p.Kp), 256, 0, s>>>(As, Ea, Ak, lda, conjA ? 0 : 2, M, M, Kc,
                                                                     (int)p.Mp, (int)p.Kp, OZT_BM, 0);
            oz_slice_tiled_kernel<<<blocks(p.Np, p.Kp), 256, 0, s>>>(Bs, Eb, Bk, ldb, 1, 2 * N, N, Kc,
                                                                     (int)p.Np, (int)p.Kp, OZT_BN, 1);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const dim3 grid((unsigned)(p.Mp / bm), (unsigned)(p.Np / OZ_BN), (unsigned)p.splits);
        cudaEvent_t ev1 = nullptr;
        if (timer) {
            cudaEvent_t ev0;
            if ((e = timer->next(&ev0)) != cudaSuccess) return e;
            if ((e = timer->next(&ev1)) != cudaSuccess) return e;
            if ((e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
        }
        if (legacy)
            oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, s>>>(As, Bs, Ea, Eb, Wp, C, ldc, M, N, (int)p.Mp,
                                                            (int)p.Np, (int)p.Kp, (int)p.kchunk,
                                                            halfN_tiles, upper ? 1 : 0, alpha, b);
        else
            oz_gemm_tc_kernel<<<grid, OZT_THREADS, OZT_SMEM, s>>>(As, Bs, Ea, Eb, Wp, C, ldc, M, N,
                                                                 (int)p.Mp, (int)p.Np, (int)p.Kp,
                                                                 (int)p.kchunk, halfN_tiles,
                                                                 upper ? 1 : 0, alpha, b, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (timer && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return e;
        if (tc_flops) *tc_flops += ozaki_tc_flops(M, N, Kc, upper, legacy);
        if (Wp) {
            oz_combine_kernel<<<grid_for((int64_t)M * N), 256, 0, s>>>(C, ldc, Wp, M, N, (int)p.Mp,
                                                                       (int)p.Np, p.splits, alpha, b,
                                                                       upper ? 1 : 0, bm);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (launches) *launches += 5 + (Wp ? 1 : 0);
    }
    if (hermitian) {  // exactly Hermitian result, whether or not tiles were skipped
        oz_mirror_kernel<<<grid_for((int64_t)M * M), 256, 0, s>>>(C, ldc, M);
        if (launches) *launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace rsrr

// ----------------------------------------------------------- C ABI
namespace rsrr {
std::string &thread_error();  // api.cu: last error of a handle-less call
}

extern "C" rsrr_status rsrr_zgemm(int32_t M, int32_t N, int32_t K, int32_t conjA, const rsrr_c128 *A,
                                  int64_t lda, const rsrr_c128 *B, int64_t ldb, rsrr_c128 *C,
                                  int64_t ldc, double alpha, double beta, int32_t method,
                                  int32_t hermitian, size_t max_ws_bytes, void *stream) {
    using namespace rsrr;
    auto fail = [](rsrr_status st, const char *what, cudaError_t e = cudaSuccess) {
        std::string m = std::string("rsrr_zgemm: ") + what;
        if (e != cudaSuccess) m += std::string(": ") + cudaGetErrorString(e);
        thread_error() = m;
        return st;
    };
    if (M < 0 || N < 0 || K < 0 || !C || (K > 0 && (!A || !B)))
        return fail(RSRR_EINVAL, "bad argument");
    const int64_t rowsA = conjA ? K : M;
    if (ldc < std::max(1, M) || ldb < std::max(1, K) || lda < std::max<int64_t>(1, rowsA))
        return fail(RSRR_EINVAL, "leading dimension too small");
    if (method < RSRR_GEMM_AUTO || method > RSRR_GEMM_OZAKI_MMA) return fail(RSRR_EINVAL, "unknown method");
    if (hermitian && (!conjA || A != B || lda != ldb || M != N || beta != 0.0))
        return fail(RSRR_EINVAL, "hermitian needs conjA, A == B, lda == ldb, M == N, beta == 0");
    cudaStream_t s = (cudaStream_t)stream;
    const double2 *a = reinterpret_cast<const double2 *>(A);
    const double2 *b = reinterpret_cast<const double2 *>(B);
    double2 *c = reinterpret_cast<double2 *>(C);
    const double flops = 8.0 * M * (double)N * K;
    const bool legacy = method == RSRR_GEMM_OZAKI_MMA;
    const bool sliced = method == RSRR_GEMM_OZAKI || legacy ||
                        (method == RSRR_GEMM_AUTO && flops >= 1073741824.0);
    cudaError_t e;
    if (!sliced) {
        if ((e = fp64_gemm(M, N, K, conjA != 0, a, lda, b, ldb, c, ldc, alpha, beta, s)) != cudaSuccess)
            return fail(RSRR_ECUDA, "fp64 gemm", e);
    } else {
        size_t need = ozaki_workspace_bytes(M, N, K, hermitian != 0);
        if (max_ws_bytes > 0) need = std::min(need, max_ws_bytes);
        // the call's own status word (bounded waits that ran out) follows the
        // slices in the same allocation
        const size_t ws_bytes = need / 256 * 256;
        void *ws = nullptr;
        if ((e = cudaMalloc(&ws, ws_bytes + 256)) != cudaSuccess) return fail(RSRR_ENOMEM, "work space", e);
        unsigned int *status = reinterpret_cast<unsigned int *>(static_cast<char *>(ws) + ws_bytes);
        unsigned int tmo = 0;
        e = cudaMemsetAsync(status, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess)
            e = ozaki_zgemm(M, N, K, conjA != 0, a, lda, b, ldb, c, ldc, alpha, beta, hermitian != 0, ws,
                            ws_bytes, s, nullptr, nullptr, nullptr, legacy, status);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&tmo, status, sizeof tmo, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && tmo != 0) {
            cudaFree(ws);
            return fail(RSRR_ETIMEOUT, "a bounded tensor-core wait ran out");
        }
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaFree(ws);
        if (e == cudaErrorMemoryAllocation) return fail(RSRR_ENOMEM, "work space below one chunk");
        if (e != cudaSuccess) return fail(RSRR_ECUDA, "sliced gemm", e);
        if (e2 != cudaSuccess) return fail(RSRR_ECUDA, "sync", e2);
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(RSRR_ECUDA, "sync", e);
    thread_error().clear();
    return RSRR_OK;
}

extern "C" rsrr_status rsrr_check_wait_timeout(int32_t tries, void *stream) {
    using namespace rsrr;
    auto fail = [](rsrr_status st, const char *msg, cudaError_t e = cudaSuccess) {
        thread_error() = e == cudaSuccess ? std::string(msg) : std::string(msg) + ": " + cudaGetErrorString(e);
        return st;
    };
    if (tries < 1 || tries > (1 << 20)) return fail(RSRR_EINVAL, "rsrr_check_wait_timeout: tries out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int *status = nullptr, tmo = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(unsigned int));
    if (e != cudaSuccess) return fail(RSRR_ECUDA, "rsrr_check_wait_timeout", e);
    e = cudaMemsetAsync(status, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        ozt_wait_check_kernel<<<1, 32, 0, s>>>((long long)tries, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tmo, status, sizeof tmo, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(status);
    if (e != cudaSuccess) return fail(RSRR_ECUDA, "rsrr_check_wait_timeout", e);
    if (tmo == 0) return fail(RSRR_OK, "rsrr_check_wait_timeout: the wait did not run out");
    return fail(RSRR_ETIMEOUT, "a bounded tensor-core wait ran out");
}
