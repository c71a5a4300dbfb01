// Trailing update of the batched dense complex64 LU on the 5th-generation
// tensor cores (RSRR step 2, Section 4.3: the factorisation of every T(z_j)).
//
// For the panel at column k0 (width jb <= 32) of every point, A22 -= L21 U12
// with L21 = rows k0+jb.. of columns k0..k0+jb-1, U12 = rows k0..k0+jb-1 of
// columns k0+jb.., A22 the trailing block; all three live in the point's
// column-major n x n complex64 matrix.
//
// Complex as one real product (the real embedding):
//   [Cr | Ci] = [Ar | Ai] [[Br, Bi], [-Bi, Br]]
// so a 128 x 128 complex output tile is a 128 x 256 real tile of depth
// K' = 64 (2 jb, zero-padded).  FP32 operands are split into TF32 parts,
// a = a_hi + a_lo (a_hi = a rounded to TF32, a_lo = the rest rounded to
// TF32), and the product is accumulated in FP32 in tensor memory as
// a_lo b_hi + a_hi b_lo + a_hi b_hi (the "3xTF32" scheme: close to FP32
// accuracy, which the FP64 refinement of the samples expects of a complex64
// factor).  Per K-step of 8 the elected thread issues three
// tcgen05.mma.kind::tf32 (M = 128, N = 256); 24 per tile.
//
// Operands are packed by all threads from global memory (L2: the panel and
// the U12 rows are read by every tile of their row / column) into shared
// memory in the K-major core-matrix layout without swizzle: per K-column of
// core matrices (4 TF32 = 16 bytes), all rows contiguous at 16 bytes a row,
// so the descriptor's SBO (next 8-row group) is 128 bytes and its LBO (next
// core matrix along K) 16 x rows bytes.  The accumulator occupies 256 columns
// of tensor memory; the epilogue reads it back (tcgen05.ld) and subtracts it
// from A22, each warp a 32-row slice (its TMEM lanes) of one half of the
// columns, a warp's 32 rows contiguous in memory for every column.
// The one mbarrier wait is bounded; a wait that runs out is counted in the
// caller's status word and the tile is left unchanged.
#include <algorithm>

#include "common.cuh"
#include "rsrr_internal.h"

namespace rsrr {
namespace tc {

constexpr int BM = 128;              // complex rows of a tile
constexpr int BN = 128;              // complex columns of a tile
constexpr int KR = 64;               // real depth (2 x 32)
constexpr int THREADS = 256;
static_assert(BM == BN && (BM * 32) % THREADS == 0, "packing: equal A and B element counts per thread");
constexpr int A_BYTES = BM * KR * 4;           // one TF32 part of A' (32 KB)
constexpr int B_BYTES = 2 * BN * KR * 4;       // one TF32 part of B' (64 KB)
constexpr size_t SMEM = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + 64;
constexpr uint32_t LBO_A = BM * 16;            // next core matrix along K (A')
constexpr uint32_t LBO_B = 2 * BN * 16;        // next core matrix along K (B')
constexpr long long WAIT_LIMIT = 1LL << 22;

// shared-memory matrix descriptor: K-major, no swizzle, start / LBO / SBO in
// 16-byte units, SBO = 128 bytes (next 8-row group), version 1
RSRR_DEV uint64_t smem_desc(uint32_t saddr, uint32_t lbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((128u >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: TF32 x TF32 -> F32, both K-major, M = 128, N = 256
RSRR_DEV uint32_t idesc_tf32_m128_n256() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
RSRR_DEV void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
RSRR_DEV void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(mbar) : "memory");
}
RSRR_DEV bool wait_parity(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
RSRR_DEV void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// a = hi + lo, both TF32 (round to nearest, ties away)
RSRR_DEV void split_tf32(float a, float &hi, float &lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(a));
    hi = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(a - hi));
    lo = __uint_as_float(l);
}
// byte offset of element (row, k) of a K-major operand with `rows` rows
RSRR_DEV uint32_t kmajor_off(int row, int k, int rows) {
    return (uint32_t)((k >> 2) * rows * 16 + row * 16 + (k & 3) * 4);
}

__global__ void __launch_bounds__(THREADS, 1)
dense_tc_update_kernel(float2 *__restrict__ A_all, int n, int k0, int jb, unsigned int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int pt = blockIdx.z;
    float2 *A = A_all + (size_t)pt * n * n;
    const int r0 = k0 + jb + blockIdx.x * BM;   // first row of the tile
    const int c0 = k0 + jb + blockIdx.y * BN;   // first column of the tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *a_hi = sm, *a_lo = sm + A_BYTES;
    unsigned char *b_hi = sm + 2 * A_BYTES, *b_lo = b_hi + B_BYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 2 * A_BYTES + 2 * B_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + 2 * A_BYTES + 2 * B_BYTES + 16);
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);

    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    // A' = [Ar | Ai]: row r, depth t (real part) and 32 + t (imaginary part).
    // Every thread first loads all its elements of A and B (32 loads in
    // flight), then splits and stores them.
    constexpr int PER = BM * 32 / THREADS;  // elements of A (and of B) per thread
    float2 va[PER], vb[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = tid + q * THREADS;
        const int t = e / BM, r = e % BM;
        va[q] = (t < jb && r0 + r < n) ? A[(size_t)(k0 + t) * n + r0 + r] : make_float2(0.f, 0.f);
        const int tb = e % 32, j = e / 32;
        vb[q] = (tb < jb && c0 + j < n) ? A[(size_t)(c0 + j) * n + k0 + tb] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = tid + q * THREADS;
        const int t = e / BM, r = e % BM;
        const float2 v = va[q];
        float h, l;
        split_tf32(v.x, h, l);
        *reinterpret_cast<float *>(a_hi + kmajor_off(r, t, BM)) = h;
        *reinterpret_cast<float *>(a_lo + kmajor_off(r, t, BM)) = l;
        split_tf32(v.y, h, l);
        *reinterpret_cast<float *>(a_hi + kmajor_off(r, 32 + t, BM)) = h;
        *reinterpret_cast<float *>(a_lo + kmajor_off(r, 32 + t, BM)) = l;
    }
    // B' rows j (real output columns) and BN + j (imaginary): depth t carries
    // (Br, Bi), depth 32 + t carries (-Bi, Br)
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = tid + q * THREADS;
        const int t = e % 32, j = e / 32;
        const float2 v = vb[q];
        float rh, rl, ih, il, nh, nl;
        split_tf32(v.x, rh, rl);
        split_tf32(v.y, ih, il);
        split_tf32(-v.y, nh, nl);
        *reinterpret_cast<float *>(b_hi + kmajor_off(j, t, 2 * BN)) = rh;
        *reinterpret_cast<float *>(b_lo + kmajor_off(j, t, 2 * BN)) = rl;
        *reinterpret_cast<float *>(b_hi + kmajor_off(j, 32 + t, 2 * BN)) = nh;
        *reinterpret_cast<float *>(b_lo + kmajor_off(j, 32 + t, 2 * BN)) = nl;
        *reinterpret_cast<float *>(b_hi + kmajor_off(BN + j, t, 2 * BN)) = ih;
        *reinterpret_cast<float *>(b_lo + kmajor_off(BN + j, t, 2 * BN)) = il;
        *reinterpret_cast<float *>(b_hi + kmajor_off(BN + j, 32 + t, 2 * BN)) = rh;
        *reinterpret_cast<float *>(b_lo + kmajor_off(BN + j, 32 + t, 2 * BN)) = rl;
    }
    // the packed operands become visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = idesc_tf32_m128_n256();
        const uint32_t ah = (uint32_t)__cvta_generic_to_shared(a_hi), al = (uint32_t)__cvta_generic_to_shared(a_lo);
        const uint32_t bh = (uint32_t)__cvta_generic_to_shared(b_hi), bl = (uint32_t)__cvta_generic_to_shared(b_lo);
#pragma unroll 1
        for (int kk = 0; kk < KR / 8; ++kk) {
            const uint32_t ao = (uint32_t)(kk * 2) * LBO_A, bo = (uint32_t)(kk * 2) * LBO_B;
            mma_tf32(tmem, smem_desc(al + ao, LBO_A), smem_desc(bh + bo, LBO_B), idesc, kk > 0 ? 1u : 0u);
            mma_tf32(tmem, smem_desc(ah + ao, LBO_A), smem_desc(bl + bo, LBO_B), idesc, 1u);
            mma_tf32(tmem, smem_desc(ah + ao, LBO_A), smem_desc(bh + bo, LBO_B), idesc, 1u);
        }
        commit(mb);
    }
    __syncwarp();
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 rows) for the
    // complex columns 64 (w / 4) .. +63: real parts in TMEM columns j, imaginary
    // parts in columns BN + j.  A22 is read 16 columns at a time into registers
    // (all 16 loads in flight together; the first group is issued before the
    // MMAs are waited for), then the product is subtracted and stored.
    const int rl = 32 * (warp & 3) + lane;
    const int cbase = 64 * (warp >> 2);
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const int row = r0 + rl;
    float2 cv[16];
    auto load_group = [&](int q) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = c0 + cbase + q + j;
            cv[j] = (row < n && c < n) ? A[(size_t)c * n + row] : make_float2(0.f, 0.f);
        }
    };
    load_group(0);
    const bool ok = wait_parity(mb, 0);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
    for (int q = 0; q < 64; q += 16) {
        float re[16], im[16];
        tmem_ld16(trow + (uint32_t)(cbase + q), re);
        tmem_ld16(trow + (uint32_t)(BN + cbase + q), im);
        if (ok && row < n) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = c0 + cbase + q + j;
                if (c < n) A[(size_t)c * n + row] = make_float2(cv[j].x - re[j], cv[j].y - im[j]);
            }
        }
        if (q + 16 < 64) load_group(q + 16);
    }
    if (!ok && lane == 0) atomicAdd(status, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
}

}  // namespace tc

cudaError_t launch_dense_tc_update(float2 *A, int n, int k0, int jb, int N, unsigned int *status,
                                   cudaStream_t s) {
    const int rest = n - k0 - jb;
    if (rest <= 0) return cudaSuccess;
    if (jb > 32 || !status) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc::dense_tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((rest + tc::BM - 1) / tc::BM), (unsigned)((rest + tc::BN - 1) / tc::BN),
                    (unsigned)N);
    tc::dense_tc_update_kernel<<<grid, tc::THREADS, tc::SMEM, s>>>(A, n, k0, jb, status);
    return cudaGetLastError();
}

}  // namespace rsrr
