// rsrr_solve_band_noalloc: one banded solve T X = U in complex128 that uses
// no allocation at all.  Its work space (band factor storage, pivots, block
// inverses, status word) lives in a fixed file-scope device array.
//
// Why: some callers cannot call cudaMalloc -- plug-ins inside a host
// application whose caching allocator or memory pool has reserved the
// device memory up front (a raw cudaMalloc would fail or fragment it), and
// latency-bound loops that must never enter the allocator.  They can still
// factor and solve one sampled system through this entry point, passing
// only their own input and output buffers.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "common.cuh"
#include "rsrr.h"
#include "rsrr_internal.h"

namespace rsrr {

// Fixed scratch: every GPU that loads the library holds these 32 MiB until the
// process exits.  All calls share it and it keeps the last call's contents.
constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::string &thread_error();  // api.cu: last error of a handle-less call

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};  // device address of the array, per device

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

rsrr_status noalloc_fail(rsrr_status st, const char *what, cudaError_t e = cudaSuccess) {
    char buf[256];
    if (e != cudaSuccess)
        snprintf(buf, sizeof buf, "rsrr_solve_band_noalloc: %s: %s", what, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof buf, "rsrr_solve_band_noalloc: %s", what);
    thread_error() = buf;
    return st;
}
}  // namespace

// Copy the caller's LAPACK band (ldb = kl+ku+1, A(i,j) at band[(ku+i-j) + j*ldb])
// into the factor layout of band_lu_kernel (A(i,j) at ab[j*ldab + kl+ku + i-j],
// ldab = 2kl+ku+NB), writing zeros everywhere else: no entry of the shared
// scratch survives from an earlier call.
__global__ void noalloc_load_band_kernel(double2 *__restrict__ ab, const double2 *__restrict__ band,
                                         int n, int kl, int ku, int ldab) {
    const int64_t total = (int64_t)ldab * n;
    const int KV = kl + ku, ldb = kl + ku + 1;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / ldab);
        const int t = (int)(idx - (int64_t)c * ldab);
        const int i = c + t - KV;
        double2 v = make_double2(0.0, 0.0);
        if (i >= 0 && i < n && i - c <= kl && c - i <= ku) v = band[(int64_t)c * ldb + (ku + i - c)];
        ab[idx] = v;
    }
}

}  // namespace rsrr

extern "C" rsrr_status rsrr_solve_band_noalloc(int64_t n, int32_t kl, int32_t ku,
                                               const rsrr_c128 *band, int32_t L,
                                               const rsrr_c128 *U, rsrr_c128 *X, void *stream) {
    using namespace rsrr;
    if (n < 1 || n > (int64_t)1 << 30 || kl < 0 || ku < 0 || L < 1 || !band || !U || !X)
        return noalloc_fail(RSRR_EINVAL, "bad argument");
    if (kl > KL_MAX) return noalloc_fail(RSRR_EINVAL, "lower bandwidth above 480");
    // band rows beyond n - 1 would hold no entry of T; they are refused rather
    // than carried through the factor storage
    if ((int64_t)kl > n - 1 || (int64_t)ku > n - 1)
        return noalloc_fail(RSRR_EINVAL, "half-bandwidths must be at most n - 1");
    const int NB = NB_C128;
    // every size in 64 bits (ku <= n - 1 < 2^30, kl <= 480, so ldab fits in int)
    const int64_t ldab = 2 * (int64_t)kl + ku + NB;
    const int64_t nblk = (n + NB - 1) / NB;
    if (ldab > (int64_t)(kNoallocScratchBytes / sizeof(double2)) / n) {
        char buf[160];
        snprintf(buf, sizeof buf, "needs more than %zu bytes of scratch, the fixed maximum is %zu",
                 kNoallocScratchBytes, kNoallocScratchBytes);
        return noalloc_fail(RSRR_EINVAL, buf);
    }
    const size_t b_ab = align256(sizeof(double2) * (size_t)ldab * (size_t)n);
    const size_t b_dinv = align256(sizeof(double2) * (size_t)nblk * 2 * NB * NB);
    const size_t b_piv = align256(sizeof(int32_t) * (size_t)n);
    const size_t b_info = align256(sizeof(int32_t));
    if (b_ab + b_dinv + b_piv + b_info > kNoallocScratchBytes) {
        char buf[160];
        snprintf(buf, sizeof buf, "needs %zu bytes of scratch, the fixed maximum is %zu",
                 b_ab + b_dinv + b_piv + b_info, kNoallocScratchBytes);
        return noalloc_fail(RSRR_EINVAL, buf);
    }
    BandGeom g;
    g.kl = kl;
    g.ku = ku;
    g.nb = NB;
    g.ldab = (int)ldab;
    // the solve's shared memory is checked before anything is launched
    if (!band_solve_fits_c128(g))
        return noalloc_fail(RSRR_EINVAL, "band too wide for the solve's shared memory");
    // device address of the scratch array on the current device, looked up by
    // the first call on that device (which should come before any stream
    // capture) and kept for the life of the process; a cudaDeviceReset
    // invalidates it, and the entry point is not usable after one
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(RSRR_ECUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(RSRR_EINVAL, "device index out of range");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return noalloc_fail(RSRR_ECUDA, "cudaGetSymbolAddress", e);
            g_noalloc_ptr[dev] = p;
        }
        base = g_noalloc_ptr[dev];
    }
    char *cp = static_cast<char *>(base);
    double2 *ab = reinterpret_cast<double2 *>(cp);
    double2 *dinv = reinterpret_cast<double2 *>(cp + b_ab);
    int32_t *piv = reinterpret_cast<int32_t *>(cp + b_ab + b_dinv);
    int32_t *info = reinterpret_cast<int32_t *>(cp + b_ab + b_dinv + b_piv);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t total = (int64_t)g.ldab * n;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    noalloc_load_band_kernel<<<grid, 256, 0, s>>>(ab, reinterpret_cast<const double2 *>(band), (int)n,
                                                   kl, ku, g.ldab);
    if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(RSRR_ECUDA, "load band", e);
    if ((e = launch_band_lu_c128(ab, piv, info, dinv, g, 1, (int)n, s)) != cudaSuccess)
        return noalloc_fail(RSRR_ECUDA, "band LU", e);
    if ((e = cudaMemcpyAsync(X, U, sizeof(double2) * (size_t)n * L, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return noalloc_fail(RSRR_ECUDA, "copy U", e);
    if ((e = launch_band_solve_c128(ab, piv, dinv, reinterpret_cast<double2 *>(X), g, 1, (int)n, L,
                                    nullptr, s)) != cudaSuccess)
        return noalloc_fail(RSRR_ECUDA, "band solve", e);
    int32_t h_info = 0;
    if ((e = cudaMemcpyAsync(&h_info, info, sizeof h_info, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return noalloc_fail(RSRR_ECUDA, "read status", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return noalloc_fail(RSRR_ECUDA, "sync", e);
    if (h_info != 0) {
        char buf[96];
        snprintf(buf, sizeof buf, "exactly zero pivot in column %d", h_info - 1);
        return noalloc_fail(RSRR_ESINGULAR, buf);
    }
    thread_error().clear();
    return RSRR_OK;
}
