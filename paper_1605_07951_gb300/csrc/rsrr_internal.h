// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <vector>
#include <stddef.h>
#include <stdint.h>

#define RSRR_MAX_TERMS_DEV 16

namespace rsrr {

// Column block of the band LU and of its solve (they must agree).
constexpr int NB_C64 = 32;
constexpr int NB_C128 = 16;
// Largest lower half-bandwidth the band kernels accept (panel rows <= 512).
constexpr int KL_MAX = 480;

// Largest opt-in dynamic shared memory per block of the current device.
// Kernels whose shared memory depends on the problem raise their limit to
// this value instead of to each launch's size: the limit belongs to the
// function, and host threads launching it with different sizes at the same
// time would otherwise overwrite each other's limit between set and launch.
inline int smem_optin_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

struct BandGeom {
    int kl, ku, nb, ldab;  // ldab = kl + ku + kl + nb
};

// Device copies of one problem (all pointers are device memory).
struct DevProblem {
    int64_t n, nnz;
    int N, L, m;
    const int32_t *row_ptr;  // n + 1 (CSR)
    const int32_t *col_idx;  // nnz
    const double *vals;      // m * nnz, term-major
    const int32_t *csc_ptr;  // n + 1 (column-major copy of the pattern)
    const int32_t *csc_row;  // nnz
    const int32_t *csc_perm; // nnz, CSC slot -> CSR entry
    const double2 *coef;     // N * m, f_i(z_j) at [j * m + i]
    const double2 *U;        // n * L probe, column major
};

// ---- band path (band.cu)
template <typename C>
cudaError_t launch_assemble(C *ab, const BandGeom &g, const DevProblem &p, cudaStream_t s);
cudaError_t launch_tnorm(double *tnorm, const DevProblem &p, cudaStream_t s);
// dinv: per point and NB block, L11^{-1} then U11^{-1} (NB x NB each)
// cluster: two CTAs per point with one-panel lookahead (band_lu.cu); the
// factors are bitwise those of the one-CTA kernel
cudaError_t launch_band_lu_c64(float2 *ab, int32_t *piv, int32_t *info, float2 *dinv,
                               const BandGeom &g, int N, int n, cudaStream_t s, bool cluster = false);
cudaError_t launch_band_lu_c128(double2 *ab, int32_t *piv, int32_t *info, double2 *dinv,
                                const BandGeom &g, int N, int n, cudaStream_t s, bool cluster = false);
// one point of one problem for the grouped band LU (ab, dinv: complex64 or
// complex128 storage of that point)
struct LuTask {
    void *ab;
    int32_t *piv, *info;
    void *dinv;
    int n, kl, ku, ldab;
};
// persistent band LU over a task list (ordered by the caller, longest first);
// *next is a zeroed device counter; kl_max the widest lower bandwidth
cudaError_t launch_band_lu_grouped_c64(const LuTask *tasks, int ntasks, int kl_max, int *next, cudaStream_t s);
cudaError_t launch_band_lu_grouped_c128(const LuTask *tasks, int ntasks, int kl_max, int *next, cudaStream_t s);
cudaError_t launch_band_solve_c64(const float2 *ab, const int32_t *piv, const float2 *dinv,
                                  float2 *B, const BandGeom &g, int N, int n, int L,
                                  const int32_t *skip, cudaStream_t s);
cudaError_t launch_band_solve_c128(const double2 *ab, const int32_t *piv, const double2 *dinv,
                                   double2 *B, const BandGeom &g, int N, int n, int L,
                                   const int32_t *skip, cudaStream_t s);
// ---- real path: real NEP at real points, real factor storage (float for
// the mixed path, double for the FP64 path), S complex with zero imaginary
// parts; the launchers mirror their complex counterparts
cudaError_t launch_band_lu_r32(float *ab, int32_t *piv, int32_t *info, float *dinv, const BandGeom &g, int N,
                               int n, cudaStream_t s, bool cluster);
cudaError_t launch_band_lu_r64(double *ab, int32_t *piv, int32_t *info, double *dinv, const BandGeom &g, int N,
                               int n, cudaStream_t s, bool cluster);
cudaError_t launch_band_solve_r32(const float *ab, const int32_t *piv, const float *dinv, float *B,
                                  const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s);
cudaError_t launch_band_solve_r64(const double *ab, const int32_t *piv, const double *dinv, double *B,
                                  const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s);
size_t band_solve2_smem_r32(const BandGeom &g);
size_t band_solve2_smem_r64(const BandGeom &g);
cudaError_t launch_band_solve2_r32(const float *ab, const int32_t *bperm, const float *dinv, float *B,
                                   const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s);
cudaError_t launch_band_solve2_r64(const double *ab, const int32_t *bperm, const double *dinv, double *B,
                                   const BandGeom &g, int N, int n, int L, const int32_t *skip, cudaStream_t s);
cudaError_t launch_broadcast_probe_r32(float *D, const double2 *U, int64_t nL, int N, cudaStream_t s);
cudaError_t launch_broadcast_probe_r64(double *D, const double2 *U, int64_t nL, int N, cudaStream_t s);
cudaError_t launch_widen_r32(double2 *X, const float *D, int64_t total, cudaStream_t s);
cudaError_t launch_widen_r64(double2 *X, const double *D, int64_t total, cudaStream_t s);
cudaError_t launch_narrow_r32(float *D, const double2 *R, int64_t per_pt, int N, const int32_t *skip,
                              cudaStream_t s);
cudaError_t launch_update_r32(double2 *X, const float *D, int64_t per_pt, int N, const int32_t *skip,
                              cudaStream_t s);
cudaError_t launch_real_part(double2 *U, int64_t total, cudaStream_t s);

// whether the one-kernel complex128 solve's shared memory (its smallest
// right-hand-side chunk) fits the device's opt-in limit for this geometry
bool band_solve_fits_c128(const BandGeom &g);
cudaError_t launch_residual(double2 *R, const double2 *X, const DevProblem &p, double *rmax,
                            double *xmax, const int32_t *skip, cudaStream_t s);
cudaError_t launch_eta(double *eta, int32_t *done, const double *rmax, const double *xmax,
                       const double *umax, const double *tnorm, int N, int L, double tol,
                       int32_t *sweep_flag, const int32_t *skip, cudaStream_t s);
cudaError_t launch_colmax(double *out, const double2 *U, int n, int L, cudaStream_t s);
cudaError_t launch_broadcast_probe_c64(float2 *D, const double2 *U, int64_t nL, int N,
                                       cudaStream_t s);
cudaError_t launch_broadcast_probe_c128(double2 *D, const double2 *U, int64_t nL, int N,
                                        cudaStream_t s);
cudaError_t launch_widen(double2 *X, const float2 *D, int64_t total, cudaStream_t s);
cudaError_t launch_narrow(float2 *D, const double2 *R, int64_t per_pt, int N, const int32_t *skip,
                          cudaStream_t s);
cudaError_t launch_update(double2 *X, const float2 *D, int64_t per_pt, int N, const int32_t *skip,
                          cudaStream_t s);

// ---- dense kernel path (dense.cu)
cudaError_t launch_assemble_dense_c64(float2 *A, const double *pts, const double2 *zs, double diag,
                                      int n, int N, cudaStream_t s);
cudaError_t launch_assemble_dense_c128(double2 *A, const double *pts, const double2 *zs, double diag,
                                       int n, int N, cudaStream_t s);
cudaError_t launch_dense_tnorm(double *tnorm, const double2 *A, int n, int N, cudaStream_t s);
// dense-terms kind: T(z_j) = sum_i coef[j m + i] A_i (A: m x n^2, term-major)
cudaError_t launch_assemble_dense_terms(double2 *T, const double2 *A, const double2 *coef, int n, int N,
                                        int m, cudaStream_t s);
// R(:, c) (+)= cf[c m + i] Y(:, c), c < cnt (first: R = ...)
cudaError_t launch_accum_term_cols(double2 *R, const double2 *Y, const double2 *cf, int m, int i, int n,
                                   int cnt, bool first, cudaStream_t s);
// squared 2-norms of the columns of R and V
cudaError_t launch_col_norms2(const double2 *R, const double2 *V, int n, int cnt, double *rr, double *vv,
                              cudaStream_t s);
// complex64 LU; tc: trailing updates on the tensor cores (3xTF32, dense_tc.cu),
// bounded waits counted in *status
cudaError_t launch_dense_lu_c64(float2 *A, int32_t *piv, int32_t *info, float2 *dinv, int n, int N,
                                cudaStream_t s, int64_t *launches, unsigned int *status, bool tc);
cudaError_t launch_dense_lu_c128(double2 *A, int32_t *piv, int32_t *info, double2 *dinv, int n, int N,
                                 cudaStream_t s, int64_t *launches);
cudaError_t launch_dense_solve_c64(const float2 *A, const int32_t *piv, const float2 *dinv, float2 *B,
                                   int n, int N, int L, const int32_t *skip, cudaStream_t s);
cudaError_t launch_dense_solve_c128(const double2 *A, const int32_t *piv, const double2 *dinv,
                                    double2 *B, int n, int N, int L, const int32_t *skip,
                                    cudaStream_t s);
cudaError_t launch_dense_colmax(const double2 *R, const double2 *X, int n, int L, double *rmax,
                                double *xmax, cudaStream_t s);
cudaError_t launch_taylor_step(double2 *A, const double *pts, double2 c, double diag, int n, int p,
                               cudaStream_t s);
cudaError_t launch_dense_eig_residual(const double2 *V, const double2 *lam, const double *pts,
                                      double diag, int n, int cnt, double *rr, double *vv, double *t1,
                                      cudaStream_t s);
cudaError_t launch_narrow_all(float2 *D, const double2 *S, int64_t total, cudaStream_t s);

// ---- streaming band solve (band_solve2.cu): composed block permutations
// (2 nb ints per block) after each LU, then the pipelined solve.  The solve
// returns cudaErrorInvalidConfiguration when its shared memory (see
// band_solve2_smem_*) exceeds 227 KB; the caller then uses launch_band_solve_*.
cudaError_t launch_block_perm(int32_t *bperm, const int32_t *piv, int n, int kl, int nb, int N,
                              cudaStream_t s);
size_t band_solve2_smem_c64(const BandGeom &g);
size_t band_solve2_smem_c128(const BandGeom &g);
// lc: right-hand sides per CTA, 16 (default), 8, 4 or 2 (more CTAs per point
// for fewer, the same operations on every column); with gate set, the launch
// runs only if *gate == want (launch_solve_gate writes it on the device)
cudaError_t launch_band_solve2_c64(const float2 *ab, const int32_t *bperm, const float2 *dinv,
                                   float2 *B, const BandGeom &g, int N, int n, int L,
                                   const int32_t *skip, cudaStream_t s, int lc = 16,
                                   const int32_t *gate = nullptr, int want = 0);
// *gate = k for the narrowest lc = 16 >> k (k = 0..3) whose CTAs for the points
// with a zero done flag fit in one wave over sms SMs, else 0
cudaError_t launch_solve_gate(const int32_t *done, int N, int L, int sms, int32_t *gate, cudaStream_t s);
cudaError_t launch_band_solve2_c128(const double2 *ab, const int32_t *bperm, const double2 *dinv,
                                    double2 *B, const BandGeom &g, int N, int n, int L,
                                    const int32_t *skip, cudaStream_t s);

// ---- column kernels of the GMRES refinement (refine.cu); column c belongs to
// point c / L, columns of points with done set are skipped
cudaError_t rf_norm(const double2 *W, int64_t n, int ncols, int L, const int32_t *done, double *out,
                    cudaStream_t s);
cudaError_t rf_dot(const double2 *V, const double2 *W, int64_t n, int ncols, int L, const int32_t *done,
                   double2 *h, cudaStream_t s);
cudaError_t rf_axpy(double2 *W, const double2 *V, const double2 *h, double sgn, int64_t n, int ncols, int L,
                    const int32_t *done, cudaStream_t s);
cudaError_t rf_scale(double2 *V, const double2 *W, const double *den, int64_t n, int ncols, int L,
                     const int32_t *done, cudaStream_t s);
cudaError_t rf_update(double2 *X, const double2 *Z, int64_t zstride, const double2 *y, int m, int64_t n,
                      int ncols, int L, const int32_t *done, cudaStream_t s);

// ---- CUDA events recorded in pairs around launches (grown on demand; api.cu)
struct EventPool {
    std::vector<cudaEvent_t> ev;
    int used = 0;
    cudaError_t next(cudaEvent_t *out);
    cudaError_t sum_pairs_ms(double *ms) const;  // sum of the recorded pairs' durations
    ~EventPool();
};

// ---- FP64 GEMM of proj.cu without split-K: C = alpha op(A) B + beta C
cudaError_t fp64_gemm(int M, int N, int K, bool conjA, const double2 *A, int64_t lda, const double2 *B,
                      int64_t ldb, double2 *C, int64_t ldc, double alpha, double beta, cudaStream_t s);

// ---- FP64-accurate complex GEMM on the bf16 tensor cores (ozaki.cu):
// C = alpha op(A) B + beta C, op(A) = A^H when conjA; hermitian (A == B,
// conjA, M == N) computes the upper block triangle and mirrors it.  ws holds
// the slices; the product is done in K chunks when ws is smaller than
// ozaki_workspace_bytes.  cudaErrorMemoryAllocation if ws cannot hold one
// chunk of 16.
// With timer set, a pair of events brackets every launch of the main kernel
// and *tc_flops grows by the tensor-core flops it issues.  The main kernel is
// the tcgen05 one; legacy selects the mma.sync kernel (kept for comparison).
// status: a device word of the caller (a handle, a request, one rsrr_zgemm
// call) into which every bounded wait of the tcgen05 kernel that ran out is
// counted; required unless legacy.  Callers zero it and read it back on their
// own stream, so a timeout in one caller's product never reaches another's.
struct EventPool;
cudaError_t ozaki_zgemm(int M, int N, int K, bool conjA, const double2 *A, int64_t lda,
                        const double2 *B, int64_t ldb, double2 *C, int64_t ldc, double alpha,
                        double beta, bool hermitian, void *ws, size_t ws_bytes, cudaStream_t s,
                        int64_t *launches, EventPool *timer = nullptr, double *tc_flops = nullptr,
                        bool legacy = false, unsigned int *status = nullptr);
size_t ozaki_workspace_bytes(int M, int N, int K, bool hermitian);
// one thread waits, with the tcgen05 kernel's bounded mbarrier wait, on a
// barrier that nothing completes; after `limit` polls the wait is counted in
// *status (failure detection without a GPU fault)
cudaError_t launch_wait_check(long long limit, unsigned int *status, cudaStream_t s);
// bf16 tensor-core flops the product issues (2 per multiply-add of slices);
// legacy: the mma.sync kernel (64-row tiles) instead of the tcgen05 kernel
double ozaki_tc_flops(int M, int N, int K, bool hermitian, bool legacy = false);

}  // namespace rsrr
