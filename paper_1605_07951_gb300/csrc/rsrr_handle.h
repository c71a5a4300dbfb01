// The handle behind rsrr_t: host descriptors, device buffers and results.
#pragma once

#include <complex>
#include <string>
#include <vector>

#include "rsrr.h"
#include "rsrr_internal.h"

namespace rsrr {

std::complex<double> eval_fn_host(const rsrr_fn &f, std::complex<double> z);
struct Handle;
// host part of rsrr_create: validation, pattern, sampling points, f_i(z_j);
// the handle holds no device memory until allocate()
rsrr_status prepare(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                    const rsrr_opts *opts, Handle **out);
// bytes of the projection stage's work space (proj.cu)
size_t projection_ws_bytes(int NL, int64_t n, int terms);
// SS-FULL moments on the GPU (ssfull_dev.cu): node chunks hold T_Q and its
// inverse for at most this many bytes; device bytes of the stage for basis k
constexpr size_t kSsfullChunkBytes = (size_t)1 << 30;
size_t ssfull_dev_bytes(int64_t k, int m, int NQ, int KQ);
std::string &thread_error();

struct Handle {
    // problem
    int64_t n = 0, nnz = 0;
    int N = 0, L = 0, m = 0, kl = 0, ku = 0;
    // the terms as held: a caller term with complex sparse values becomes two,
    // Re A_u with f_u and Im A_u with i f_u (fn_imag marks the second)
    std::vector<rsrr_fn> fn;
    std::vector<int> fn_src;          // caller term of each held term
    std::vector<char> fn_imag;        // held term is the imaginary part of its caller term
    std::vector<double> a1;           // ||A_u||_1 of the caller's terms (residual scale)
    rsrr_fn_callback cb = nullptr;    // RSRR_F_CALLBACK terms
    void *cb_user = nullptr;
    uint64_t seed = 0;                // default probe
    bool points_added = false;        // rsrr_add_points ran: the points are explicit
    bool rect_gl = false;             // rectangle with Gauss-Legendre sampling points
    // band factor storage (factors, block inverses and permutations, residual
    // and correction buffers) holds fcap points; with fcap < N
    // (RSRR_FLAG_CHUNK_POINTS) the points are sampled in chunks of fcap and
    // the storage starts at point fbase of the chunk being sampled
    int fcap = 0, fbase = 0;
    bool chunked() const { return fcap < N; }
    int64_t fo(int p0) const { return (int64_t)p0 - fbase; }
    rsrr_region region = {};
    rsrr_opts opts = {};
    BandGeom geom = {};
    DevProblem dp = {};
    std::vector<std::complex<double>> z;
    std::vector<int32_t> h_row_ptr, h_col_idx, h_csc_ptr, h_csc_row, h_csc_perm;
    std::vector<double> h_vals;
    // dense problems: the Helmholtz kernel, or caller-supplied dense terms
    bool dense = false;
    bool dense_terms = false;         // T = sum_i f_i A_i with dense A_i (RSRR_NEP_DENSE)
    std::vector<double2> h_Aterms;    // m x n^2 host copy, dropped after the upload
    double2 *d_Aterms = nullptr;      // m x n^2 on the device
    double diag = 0.0;
    std::vector<double> h_points;
    double *d_points = nullptr;       // 3n
    double2 *d_z = nullptr;           // N sampling points
    double2 *d_T64 = nullptr;         // N dense complex128 matrices (residuals)
    float2 *d_A32 = nullptr;          // N dense complex64 factors
    void *d_dws = nullptr;            // slices of the residual products T X (Ozaki)
    size_t dws_bytes = 0;
    // device buffers (owned)
    std::vector<void *> allocations;
    size_t device_bytes = 0;
    // A handle run by the request server draws its memory from a stream-ordered
    // pool on its own stream `hs`, and every internal copy and wait goes to
    // `hs`, so that requests on other streams keep running.  With hs == NULL
    // (rsrr_create) memory comes from cudaMalloc and waits are device-wide.
    cudaStream_t hs = nullptr;
    cudaMemPool_t pool = nullptr;
    bool dry = false;                 // alloc() only counts bytes (estimates)
    std::vector<double2> h_coef;      // f_i(z_j), N x m, kept until allocate()
    int32_t *d_row_ptr = nullptr, *d_col_idx = nullptr;
    int32_t *d_csc_ptr = nullptr, *d_csc_row = nullptr, *d_csc_perm = nullptr;
    double *d_vals = nullptr;
    double2 *d_coef = nullptr, *d_U = nullptr;
    double *d_umax = nullptr;
    double2 *d_X = nullptr;           // S = [X_0 ... X_{N-1}], n x NL
    double2 *d_R = nullptr;           // FP64 residuals (mixed path)
    float2 *d_D = nullptr;            // complex64 corrections (mixed path)
    // real path (RSRR_FLAG_REAL: real NEP at real points): real factors, block
    // inverses and corrections; S stays complex with zero imaginary parts
    bool real = false;
    float *d_abr32 = nullptr, *d_dinvr32 = nullptr, *d_Dr32 = nullptr;
    double *d_abr64 = nullptr, *d_dinvr64 = nullptr, *d_Dr64 = nullptr;
    float2 *d_ab32 = nullptr;         // complex64 band factors
    double2 *d_ab64 = nullptr;        // complex128 band factors
    float2 *d_dinv32 = nullptr;       // per block L11^{-1}, U11^{-1} (complex64)
    double2 *d_dinv64 = nullptr;      // per block L11^{-1}, U11^{-1} (complex128)
    int32_t *d_piv = nullptr, *d_info = nullptr, *d_done = nullptr, *d_sweep_flags = nullptr;
    int32_t *d_bperm = nullptr;       // composed row permutation of every block (streaming solve)
    int32_t *d_gate = nullptr;        // shape of a refinement sweep's solve (few points left: narrow)
    // GMRES refinement (allocated on first use): Krylov vectors V_0..V_m and
    // preconditioned directions Z_0..Z_{m-1} (n x N L each), zero probe, the
    // per-column Hessenberg entries, norms and coefficients
    double2 *d_gV = nullptr, *d_gZ = nullptr, *d_zeroU = nullptr, *d_gH = nullptr, *d_gy = nullptr;
    double *d_gnorm = nullptr;
    size_t gmres_bytes = 0;
    bool solve2 = false;              // streaming band solve possible (block permutations allocated)
    bool use_solve2 = false;          // streaming band solve in use (autotuned or solve2)
    bool cluster_lu = true;           // band LU by a cluster of two CTAs per point
    bool tuned = false;               // the autotuner's choice is applied
    // CUDA graph of rsrr_sample (RSRR_FLAG_GRAPH, band path)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;
    int graph_calls = 0;
    bool graph_failed = false;
    double *d_tnorm = nullptr, *d_eta = nullptr, *d_rmax = nullptr, *d_xmax = nullptr;

    // projection stage (proj.cu)
    int k = 0, kc = 0;
    double sigma1 = 0.0, sigmak = 0.0;
    double2 *d_Q = nullptr;           // n x k basis
    double2 *d_P = nullptr;           // m blocks of k x k
    void *proj_ws = nullptr;          // projection work space (allocated on first use)
    size_t proj_ws_bytes = 0;

    // results of rsrr_solve
    std::vector<rsrr_c128> res_lam, res_V;
    std::vector<double> res_res;

    // state
    bool sampled = false, projected = false, solved = false;
    int stat_sweeps = 0, stat_converged = 0, stat_singular = -1;
    double stat_max_eta = 0.0;
    std::string err;
    int64_t launches = 0;
    cudaEvent_t events[8] = {};
    bool timed_sample = false, timed_project = false;
    // device word counting the bounded tensor-core waits that ran out in this
    // handle's products since its last rsrr_sample (zeroed there, read by rsrr_solve)
    unsigned int *d_tmo = nullptr;
    double stage_ms[6] = {};
    // GEMM timing of the last rsrr_project (opts.timing)
    EventPool gemm_pool;                // pairs around every product
    EventPool tc_pool;                  // pairs around the sliced products' main kernel
    double gemm_flops = 0.0, gemm_ms = 0.0;
    double tc_flops = 0.0, tc_ms = 0.0;
    bool gemm_timed = false;

    ~Handle();
    cudaError_t gemm_event(cudaEvent_t *out);
    rsrr_status fail(rsrr_status st, const char *what, cudaError_t e = cudaSuccess);
    template <typename T> cudaError_t alloc(T **p, size_t count);
    cudaError_t raw_alloc(void **p, size_t bytes);
    cudaError_t raw_free(void *p);
    void release(void *p, size_t bytes);
    template <typename T> cudaError_t regrow(T **p, size_t per, int N0, int N1, bool keep);
    cudaError_t wait();
    rsrr_status allocate();
    size_t estimate_bytes();
    rsrr_status allocate_and_upload(const std::vector<double2> &coef);
    rsrr_status sample(cudaStream_t s);  // every point, band or dense
    rsrr_status sample_graph(cudaStream_t s);
    rsrr_status autotune(cudaStream_t s);
    void drop_graph();
    // phase 0: everything; 1: up to the assembly (the caller factors); 2: from
    // after the LU (the caller factored)
    rsrr_status sample_band(int p0, int np, cudaStream_t s, int phase = 0);
    // points p0 .. p0+np-1 through sample_band, chunk by chunk when chunked()
    rsrr_status sample_range(int p0, int np, cudaStream_t s);
    // GMRES refinement cycles of points p0 .. p0+np-1 (mixed band path)
    rsrr_status refine_gmres(int p0, int np, const DevProblem &dq, cudaStream_t s);
    cudaError_t band_solve(bool mixed, void *B, const int32_t *skip, int p0, int np, cudaStream_t s);
    // the real path's solve of points p0 .. p0+np-1 (float or double B)
    cudaError_t real_solve(bool mixed, void *B, const int32_t *skip, int p0, int np, cudaStream_t s);
    // a refinement sweep's complex64 solve: streaming solve in the wide shape
    // while many points are left, in the narrow one when few are (chosen on
    // the device from the done flags)
    cudaError_t sweep_solve(float2 *B, const int32_t *skip, int p0, int np, cudaStream_t s);
    rsrr_status sample_dense(int p0, int np, cudaStream_t s);
    rsrr_status dense_residual(bool skip_done, int p0, int np, cudaStream_t s);
    // appends sampling points (buffers regrown, the old samples kept) and
    // samples only the new ones
    rsrr_status add_points(const std::complex<double> *znew, int count, cudaStream_t s);
    bool dense_residual_sliced() const;
    rsrr_status allocate_dense();
    rsrr_status read_outcome();
    rsrr_status mark(int i, cudaStream_t s);
    rsrr_status project(cudaStream_t s);
    rsrr_status solve(rsrr_result *out);
    // f of every held term at count points (point-major, count x fn.size());
    // EINVAL if a value is not finite
    rsrr_status eval_terms(const std::complex<double> *z, int64_t count,
                           std::vector<std::complex<double>> &out);
    // sum over the caller's terms of |f_u(lam)| ||A_u||_1, from held-term values
    double residual_scale(const std::complex<double> *f_held) const;
    // weights of the moment methods at the sampling points
    void moment_weights(std::vector<std::complex<double>> &w) const;
    // nodes and weights dz/(2 pi) of the contour integrals of SS-FULL: the
    // trapezoid rule on the ellipse or composite Gauss on the rectangle
    void contour_quadrature(int NQ, std::vector<std::complex<double>> &zq,
                            std::vector<std::complex<double>> &wq) const;
    bool inside(std::complex<double> z) const;  // strict interior of the contour
    // SS-RI on the samples (rsrr_solve with RSRR_METHOD_SS_RI): eigenvalues
    // and the sample-space coefficients ZWB (N L x nbar) of v = S ZWB
    rsrr_status ss_ri(cudaStream_t s, std::vector<std::complex<double>> &lam,
                      std::vector<std::complex<double>> &ZWB, int &nbar, double &gmax);
    rsrr_status ssfull_moments(const std::vector<std::complex<double>> &fq,
                               const std::vector<std::complex<double>> &zq,
                               const std::vector<std::complex<double>> &wq, int KQ,
                               std::vector<std::vector<std::complex<double>>> &Am);
};

}  // namespace rsrr
