/*
 * rsrr.h -- C ABI of the GB300 resolvent-sampling library.
 *
 * The library computes the data-parallel part of the resolvent sampling based
 * Rayleigh-Ritz method (RSRR) of Xiao, Zhang, Huang and Sakurai (2016) for a
 * nonlinear eigenvalue problem T(lambda) v = 0 with
 *
 *     T(z) = sum_{i<m} f_i(z) A_i                         (Eq. 1, Section 2.1)
 *
 * where the A_i are real n x n matrices sharing one sparse (banded) pattern
 * and the f_i are scalar functions.  The steps are those of the RSRR
 * algorithm in Section 4.3:
 *
 *   rsrr_create   step 1: sampling points z_j, coefficient table f_i(z_j),
 *                 device copies of the pattern and values.
 *   rsrr_sample   step 2: X_j = T(z_j)^{-1} U for every point (assembly,
 *                 banded LU with partial pivoting, triangular solves and FP64
 *                 iterative refinement), all on the GPU.
 *   rsrr_project  steps 3-4 (GPU part): S = [X_0 ... X_{N-1}] with unit-norm
 *                 columns (Section 4.2, last paragraph), orthonormal basis Q of
 *                 its dominant singular subspace (Section 4.3 step 3), and the
 *                 projected coefficients P_i = Q^H A_i Q (Section 4, T_Q).
 *   rsrr_solve    steps 4-5 (host part): the projected NEP by SS-FULL
 *                 (Section 3.3 with U = I), eigenvectors v = Q g and their
 *                 residuals.
 *
 * Conventions.
 *   - Complex numbers are rsrr_c128 {re, im}, layout compatible with C99
 *     double _Complex, std::complex<double> and torch.complex128.
 *   - Matrices are column major.
 *   - Host pointers are plain CPU memory; device pointers are CUDA device
 *     memory of the current device.  Which one an argument is, is stated.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL is the
 *     legacy default stream).
 *   - Every call returns an rsrr_status.  Negative values are errors, 0 is
 *     success, positive values are warnings.  No C++ exception crosses the ABI.
 *     rsrr_last_error() gives a one-line description of the last failure.
 *   - A handle is used by one host thread at a time; distinct handles are
 *     independent.  The handle owns all device memory it allocates; inputs
 *     are copied at rsrr_create and may be freed by the caller on return.
 */
#ifndef RSRR_H
#define RSRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double re, im;
} rsrr_c128;

typedef enum {
    RSRR_OK = 0,
    RSRR_EINVAL = -1,    /* invalid argument or descriptor */
    RSRR_ENOMEM = -2,    /* device or host allocation failed */
    RSRR_ESINGULAR = -3, /* an exactly zero pivot: a sampling point on an eigenvalue */
    RSRR_ENOCONV = -4,   /* refinement did not reach eta_tol for every column */
    RSRR_ETIMEOUT = -5,  /* a bounded device-side wait ran out */
    RSRR_ECUDA = -6,     /* a CUDA runtime error */
    RSRR_ESTATE = -7,    /* call out of order (e.g. rsrr_project before rsrr_sample) */
    RSRR_WGAP = 1        /* warning: the gap test g_max >= tol_gap failed (Section 3.3) */
} rsrr_status;

/* Scalar coefficient functions f(z) = scale * base(z) (the families of
 * Section 2.1; EXP covers delay problems, TAYLOR the power basis of an
 * expanded T, CALLBACK any f the caller can evaluate, Section 4.3 notes that
 * the method only needs T at the sampling points):
 *   RSRR_F_ONE       base = 1
 *   RSRR_F_ZPOW      base = z^param, param a non-negative integer
 *   RSRR_F_RATIONAL  base = z / (z - param)
 *   RSRR_F_INV       base = 1 / (param - z)
 *   RSRR_F_SQRT      base = sqrt(z^2 - param^2), principal branch
 *   RSRR_F_EXP       base = exp(-param z)
 *   RSRR_F_TAYLOR    base = (z - shift)^power, power a non-negative integer
 *   RSRR_F_CALLBACK  base = the value rsrr_nep.callback returns for this term
 *                    (it is asked for whole arrays of points at once)        */
enum {
    RSRR_F_ONE = 0,
    RSRR_F_ZPOW = 1,
    RSRR_F_RATIONAL = 2,
    RSRR_F_INV = 3,
    RSRR_F_SQRT = 4,
    RSRR_F_EXP = 5,
    RSRR_F_TAYLOR = 6,
    RSRR_F_CALLBACK = 7
};

typedef struct {
    int32_t kind;
    int32_t power;     /* RSRR_F_TAYLOR: the exponent (0 .. 64) */
    double param;
    rsrr_c128 scale;
    rsrr_c128 shift;   /* RSRR_F_TAYLOR: the expansion point */
} rsrr_fn;

/* Host callback for RSRR_F_CALLBACK terms: writes base_term(z[q]) into out[q]
 * for q < count.  It is called by rsrr_create / rsrr_describe /
 * rsrr_estimate_bytes (at the sampling points), rsrr_add_points (at the new
 * points) and rsrr_solve (at the quadrature nodes and at the eigenvalues),
 * on the calling thread or, for the request server, on a worker thread.  It
 * and `user` must stay valid until the handle is destroyed; it must return
 * finite values at every point it is asked for. */
typedef void (*rsrr_fn_callback)(int32_t term, const rsrr_c128 *z, int64_t count, rsrr_c128 *out,
                                 void *user);

#define RSRR_MAX_TERMS 8

/* The NEP.  Three kinds:
 *
 * RSRR_NEP_SPARSE: T(z) = sum_{i<m} fn[i](z) A_i.  All A_i share one CSR
 * pattern (row_ptr, col_idx; columns need not be sorted; duplicates are not
 * allowed); their values are stored term-major: A_i's value for pattern
 * entry e is values[i * nnz + e], nnz = row_ptr[n], real doubles, or
 * rsrr_c128 when values_complex is nonzero (values then points to 2 m nnz
 * doubles).  The half-bandwidths kl, ku are detected from the pattern
 * (kl <= 480) and the band path is used.  A term with complex values is held
 * as two real terms, Re A_i with fn[i] and Im A_i with i fn[i]; the
 * statistics and rsrr_get_projected count terms that way.
 *
 * RSRR_NEP_HELMHOLTZ: the dense Nystrom single-layer kernel of Section 2.1,
 * T(z)_ij = exp(i z r_ij) / (4 pi r_ij) for i != j and T_ii = diag, with
 * r_ij the distances between the n points (points[3i..3i+2], row major);
 * m, fn and the CSR fields are ignored.  The dense path is used, and the
 * projection expands T in a Taylor series about the region centre
 * (Section 6 interpolates T for the same purpose).
 *
 * RSRR_NEP_DENSE: T(z) = sum_{i<m} fn[i](z) A_i with caller-supplied dense
 * complex A_i (dense[i]: n x n, column major, n <= 32768) -- a general
 * "black-box" T such as the BEM matrices of Section 2.1 with their
 * dependence on z separated into known functions.  The dense path is used;
 * P_i = Q^H A_i Q.
 *
 * All arrays are host memory and are copied by rsrr_create. */
enum { RSRR_NEP_SPARSE = 0, RSRR_NEP_HELMHOLTZ = 1, RSRR_NEP_DENSE = 2 };

typedef struct {
    int64_t n;
    int32_t m;    /* 1 <= m <= RSRR_MAX_TERMS (sparse and dense kinds) */
    int32_t kind; /* RSRR_NEP_SPARSE, RSRR_NEP_HELMHOLTZ or RSRR_NEP_DENSE */
    const int64_t *row_ptr; /* host, n + 1 */
    const int32_t *col_idx; /* host, nnz */
    const double *values;   /* host, m * nnz (real) or 2 * m * nnz (values_complex) */
    rsrr_fn fn[RSRR_MAX_TERMS];
    const double *points;   /* host, 3n (Helmholtz kind) */
    double diag;            /* T_ii (Helmholtz kind) */
    int32_t values_complex; /* sparse kind: values are rsrr_c128 */
    int32_t reserved;
    const rsrr_c128 *const *dense; /* host, m pointers to n x n column-major A_i (dense kind) */
    rsrr_fn_callback callback;     /* for RSRR_F_CALLBACK terms */
    void *callback_user;           /* passed to callback */
} rsrr_nep;

/* Region.  For every kind but RSRR_REGION_RECT the ellipse
 * phi(t) = center + a cos t + i b sin t is the contour of the projected
 * solve (N_Q-point trapezoid rule, Eq. 58) and defines "inside".  Sampling
 * points are the N-point trapezoid nodes z_j = phi(2 pi (j + 1/2)/N) (Eq. 58,
 * Section 5.1) for RSRR_REGION_ELLIPSE, the N given host points for
 * RSRR_REGION_POINTS (the rational interpolation approach lets them lie
 * anywhere, Section 3.3), or, for RSRR_REGION_INTERVAL, the N Chebyshev
 * points of the first kind z_i = center + a cos((2i + 1) pi / 2N) (Eq. 42) on
 * the ellipse's major axis (an interval of interest of a real NEP, Sections
 * 3.3 and 5.1).
 *
 * RSRR_REGION_RECT (Section 5.4): the rectangle with vertices
 * center +- a +- i b is the contour and the region (strict interior).
 * Sampling points: Gauss-Legendre nodes on its sides, counterclockwise from
 * the lower-left vertex -- nx on each side parallel to the real axis and
 * ny = N/2 - nx on each of the other two (N even, 1 <= nx <= N/2 - 1; the
 * paper's 27 and 13 for N = 80) -- or, when points is not NULL, the N given
 * points.  The contour integrals of SS-FULL use composite Gauss quadrature:
 * side s of length len_s is cut into max(1, round(N_Q len_s / (10 perimeter)))
 * equal panels with the 10-point Gauss-Legendre rule each (about N_Q nodes).
 * The moment weights of SS-RI and SSRR-M at the Gauss-Legendre sampling
 * points are the contour weights dz/(2 pi). */
enum { RSRR_REGION_ELLIPSE = 0, RSRR_REGION_POINTS = 1, RSRR_REGION_INTERVAL = 2, RSRR_REGION_RECT = 3 };

typedef struct {
    int32_t kind;
    int32_t nx;               /* RSRR_REGION_RECT: points per horizontal side */
    rsrr_c128 center;
    double a, b;              /* semi-axes (half-widths for the rectangle) along the
                                 real and imaginary axis, > 0 */
    const rsrr_c128 *points;  /* host, N: RSRR_REGION_POINTS, or RSRR_REGION_RECT's
                                 explicit points (NULL: Gauss-Legendre nodes) */
} rsrr_region;

/* Precision of the factorisation.
 *   RSRR_PREC_FP64   complex128 LU and solve, one residual pass for the
 *                    statistics, no refinement ("plain FP64 path").
 *   RSRR_PREC_MIXED  complex64 LU and solves on the GPU, refined to FP64
 *                    accuracy: r = U - T(z_j) X in FP64, d = LU \ r in
 *                    complex64, X += d, until every column's backward error
 *                    eta = ||r||_inf / (||T||_inf ||x||_inf + ||u||_inf) is
 *                    <= eta_tol or max_refine sweeps have run.            */
enum { RSRR_PREC_FP64 = 0, RSRR_PREC_MIXED = 1 };

/* Arithmetic of the projection's dense complex products (Gram matrices of S,
 * Q^H R, R W, Q^H A_i Q; Section 4.3's orthonormalisation and projection).
 *   RSRR_GEMM_FP64   native FP64 fused multiply-adds.
 *   RSRR_GEMM_OZAKI  FP64-accurate products on the bf16 tensor cores: both
 *                    operands are scaled per row / column by powers of two,
 *                    rounded to 55-bit fixed point and split into 7 signed
 *                    8-bit slices; slice products are summed exactly in FP32
 *                    groups and combined in 64-bit integers (Ozaki scheme).
 *                    Error per entry below 2^-52 max|a_i.| max|b_.j| K.
 *                    The slice products run on the 5th-generation tensor
 *                    cores (tcgen05.mma, accumulators in tensor memory).
 *   RSRR_GEMM_OZAKI_MMA  the same slices with the warp-level mma.sync
 *                    instructions instead (kept for comparison).
 *   RSRR_GEMM_AUTO   OZAKI for products of at least 2^30 flops, else FP64. */
enum { RSRR_GEMM_AUTO = 0, RSRR_GEMM_FP64 = 1, RSRR_GEMM_OZAKI = 2, RSRR_GEMM_OZAKI_MMA = 3 };

/* RSRR_FLAG_PLAIN_SOLVE: banded solves of rsrr_sample by the one-kernel
 * solve (factor panels read straight from global memory) instead of the
 * streaming solve; same arithmetic, kept for comparison and as the fallback
 * for bands too wide for the streaming solve's shared-memory window. */
/* RSRR_FLAG_ONE_CTA_LU: band LU of rsrr_sample by one CTA per sampling point
 * instead of a cluster of two CTAs per point (the second CTA updates most of
 * the trailing window while the first factors the next panel); the factors
 * are bitwise the same, the flag exists for comparison. */
/* RSRR_FLAG_INJECT_TIMEOUT: failure detection without a GPU fault.
 * rsrr_sample also runs one bounded device wait on a barrier that nothing
 * completes (a few thousand polls); the wait runs out and is counted in this
 * handle's own status word, exactly like a timed-out wait of its tensor-core
 * products, so rsrr_solve returns RSRR_ETIMEOUT.  Nothing else changes.  It
 * exists to test that a timeout stays with the request that met it. */
/* RSRR_FLAG_SIMT_DENSE_UPDATE: the trailing updates of the dense complex64 LU
 * (Helmholtz and dense kinds, mixed precision) on FP32 FMAs instead of the
 * tensor cores (tcgen05, 3xTF32); kept for comparison. */
enum {
    RSRR_FLAG_PLAIN_SOLVE = 1,
    RSRR_FLAG_ONE_CTA_LU = 2,
    RSRR_FLAG_INJECT_TIMEOUT = 4,
    RSRR_FLAG_SIMT_DENSE_UPDATE = 8,
    RSRR_FLAG_GRAPH = 16,
    RSRR_FLAG_AUTOTUNE = 32,
    RSRR_FLAG_WIDE_SOLVE_ONLY = 64,
    RSRR_FLAG_REAL = 128,
    RSRR_FLAG_CHUNK_POINTS = 256
};
/* RSRR_FLAG_CHUNK_POINTS (band path, with mem_budget_bytes > 0): when the
 * handle would exceed the budget, rsrr_create sizes the band factor storage
 * (factors, block inverses and permutations, residual and correction
 * buffers) for as many sampling points as fit, and rsrr_sample factors,
 * solves and refines the points chunk by chunk through that storage; S, the
 * backward errors and everything after sampling are those of the whole
 * handle (the factors of a point are not kept after its chunk).  ENOMEM only
 * if not even one point fits.  Such a handle is refused by
 * rsrr_sample_batch; RSRR_FLAG_AUTOTUNE is ignored. */
/* RSRR_FLAG_REAL: real arithmetic for a real NEP at real sampling points
 * (Sections 3.3 and 5.1: real points, e.g. the Chebyshev points of an
 * RSRR_REGION_INTERVAL, keep T(z_j) real and halve the time and memory of
 * the solves).  Requires the sparse kind with real values, real sampling
 * points and real f_i there (rsrr_create checks all three, EINVAL
 * otherwise).  The band factors, block inverses and corrections are real
 * (float for the mixed path, double for the FP64 path); the probe U is real
 * (imaginary parts of a given U are dropped); the samples S are stored as
 * complex numbers with zero imaginary parts, so the FP64 residuals, the
 * projection and rsrr_get_samples are those of the complex path.
 * RSRR_REFINE_GMRES with it is refused by rsrr_create (EINVAL), as are
 * rsrr_add_points and rsrr_sample_batch on such a handle; RSRR_FLAG_AUTOTUNE
 * is ignored. */
/* RSRR_FLAG_WIDE_SOLVE_ONLY: the refinement sweeps' streaming solves always
 * take 16 right-hand sides per CTA.  By default a sweep in which few points
 * are still above eta_tol (the points next to an eigenvalue converge last)
 * runs a narrow shape instead, 4 right-hand sides per CTA and so four times
 * as many CTAs per point, which shortens the per-point chain of block
 * solves; the shape is chosen on the device from the points' done flags, so
 * the sweeps stay asynchronous.  Both shapes do the same operations on every
 * column (bit for bit the same samples); the flag exists for comparison. */
/* RSRR_FLAG_GRAPH: rsrr_sample of the band path replays a CUDA graph: the
 * first call runs eagerly, the second captures the call's launches on the
 * caller's stream (it must not be the legacy default stream) and launches the
 * graph, later calls launch it again (one launch in place of about 5 per
 * refinement sweep).  If capture is not possible the call runs eagerly.
 * rsrr_add_points drops the graph (buffers move).
 * RSRR_FLAG_AUTOTUNE: the first rsrr_sample of the band path times the band
 * LU as a cluster of two CTAs per point and as one CTA per point, and the
 * streaming and the one-kernel solve, on the handle's own data, keeps the
 * faster of each (results agree: the LU variants bitwise, the solves to
 * rounding before refinement) and caches the choice per shape (n, kl, ku, N,
 * L, precision) for the rest of the process; that first call waits for its
 * timings. */

typedef struct {
    int32_t precision;   /* RSRR_PREC_MIXED by default */
    int32_t max_refine;  /* refinement sweeps, default 8 */
    double eta_tol;      /* default 1e-10 */
    double delta;        /* SVD truncation of S relative to sigma_1, paper's 1e-14 */
    double delta_floor;  /* resolution floor of the Gram-based SVD relative to sigma_1;
                            <= 0 (default): for RSRR the samples' accuracy --
                            0.1 eta_tol for the mixed path (1e-11), 1e-12 for
                            the FP64 path; 1e-12 for SSRR-M, whose high moments
                            carry eigen-directions far below sigma_1 of M */
    double tol_gap;      /* gap test of SS-FULL, default 1e3 (Section 3.3) */
    double res_tol;      /* acceptance of an eigenpair by residual, default 1e-6 */
    int32_t NQ;          /* SS-FULL quadrature points, default 500 */
    int32_t KQ;          /* SS-FULL moments, default 2 */
    int32_t host_threads;/* threads of rsrr_solve, 0 = all cores */
    int32_t timing;      /* nonzero: record CUDA events around every stage on the
                            caller's stream; times appear in rsrr_stats.stage_ms */
    int32_t gemm;        /* RSRR_GEMM_AUTO by default */
    int32_t flags;       /* RSRR_FLAG_* bits, 0 by default */
    uint64_t seed;       /* seed of the default probe U (complex normal entries from
                            a splitmix64 stream); rsrr_set_probe replaces U */
    int64_t mem_budget_bytes; /* > 0: rsrr_create refuses (ENOMEM) a handle whose
                            rsrr_estimate_bytes exceed it, or with
                            RSRR_FLAG_CHUNK_POINTS samples the points in chunks
                            that fit; 0 (default): no limit */
    int32_t method;      /* RSRR_METHOD_*, default RSRR_METHOD_RSRR */
    int32_t K;           /* moments of SSRR-M and SS-RI (1 <= K <= N), default 2 */
    int32_t refine;      /* RSRR_REFINE_*, default RSRR_REFINE_IR (band path, mixed precision) */
    int32_t gmres_m;     /* Krylov steps per GMRES cycle (1 .. 16), default 4 */
    int32_t chunk_points;/* band path: > 0 holds the band factor storage of at most
                            this many points and samples the points in chunks of
                            that many (as RSRR_FLAG_CHUNK_POINTS does to fit a
                            budget); 0 (default): all N points at once */
    int32_t reserved;
} rsrr_opts;

/* Refinement of the mixed-precision samples (band path):
 *   RSRR_REFINE_IR     r = U - T X in FP64, d = LU \ r in complex64, X += d,
 *                      sweeps queued asynchronously (the default).
 *   RSRR_REFINE_GMRES  each of the max_refine cycles computes r = U - T X in
 *                      FP64 and runs gmres_m steps of GMRES on T d = r per
 *                      column, right-preconditioned by the complex64 LU
 *                      (Arnoldi vectors and products in FP64, modified
 *                      Gram-Schmidt on the GPU, the small least-squares
 *                      problems on the host), then X += d; robust where
 *                      T(z_j) is too ill-conditioned for plain refinement
 *                      (points close to eigenvalues).  It waits for the
 *                      stream once a cycle and holds (2 gmres_m + 1) n N L
 *                      complex128 of Krylov vectors, allocated on first use. */
enum { RSRR_REFINE_IR = 0, RSRR_REFINE_GMRES = 1 };

/* Method of rsrr_project / rsrr_solve on the same samples X_j:
 *   RSRR_METHOD_RSRR    the resolvent sampling scheme (Section 4.3): basis of
 *                       S = [X_0 ... X_{N-1}].
 *   RSRR_METHOD_SSRR_M  the resolvent moment scheme (Section 4.1): basis of
 *                       M = [M_0 ... M_{K-1}], M_a = sum_i w_i s_i^a X_i (Eq. 40,
 *                       Eq. 48), then the same projection and SS-FULL.
 *   RSRR_METHOD_SS_RI   SS-RI (Section 3.3): moments A_a = sum_i w_i s_i^a U^H X_i
 *                       (Eq. 18), the Hankel pencil H^< - lambda H (Eq. 33) by
 *                       truncated SVD and the gap test (Eq. 44), eigenvectors
 *                       v = M W0 Sigma0^{-1} b (Eq. 41); rsrr_project does
 *                       nothing for it and rsrr_solve follows rsrr_sample.
 * s_i = (z_i - center) / max(a, b) (a fixed change of polynomial basis that
 * keeps the pencil's eigenvalues and span(M)); the weights w_i are the
 * trapezoid weights (1/N) phi'(alpha_i) of Eq. 58 on the ellipse, the
 * Chebyshev weights (-1)^i sin((2i + 1) pi / 2N) of Eq. 43 on an interval,
 * and the scaled barycentric weights of Eq. 19 for explicit points.  Both
 * moment methods are kept for comparison (Sections 5.1, 5.2). */
enum { RSRR_METHOD_RSRR = 0, RSRR_METHOD_SSRR_M = 1, RSRR_METHOD_SS_RI = 2 };

typedef struct rsrr_handle rsrr_t;

typedef struct {
    int64_t n;
    int32_t N, L, m, kl, ku;
    int32_t refine_sweeps; /* sweeps run by the last rsrr_sample */
    int32_t converged;     /* 1 if every column reached eta_tol */
    int32_t singular_point;/* first point with an exactly zero pivot, or -1 */
    int32_t k;             /* rank kept by the last rsrr_project */
    int32_t kc;            /* columns kept by its pivoted Cholesky stage */
    double max_eta;        /* largest per-column backward error after rsrr_sample
                              (NaN if one is not finite or could not be read back) */
    double sigma1, sigmak; /* largest and smallest kept singular value of S */
    size_t device_bytes;   /* device memory held by the handle */
    int64_t launches;      /* CUDA kernels launched by the handle since rsrr_create */
    /* with opts.timing: device time (ms) of the last rsrr_sample / rsrr_project
     * stages: [0] assembly + ||T||, [1] band LU, [2] first solve, [3] refinement
     * sweeps, [4] final backward errors, [5] rsrr_project */
    double stage_ms[6];
    /* with opts.timing, for the last rsrr_project: algorithmic flops of its
     * FP64 GEMMs (8 per complex multiply-add, unique entries only for the
     * Hermitian products) and their summed device time */
    double gemm_flops, gemm_ms;
    /* with opts.timing, for the last rsrr_project: bf16 tensor-core flops
     * issued by the sliced (RSRR_GEMM_OZAKI) products' main kernel and the
     * summed device time of that kernel alone */
    double tc_flops, tc_ms;
} rsrr_stats;

/* Result of rsrr_solve.  Arrays are host memory owned by the handle, valid
 * until the next rsrr_solve or rsrr_destroy. */
typedef struct {
    int32_t count;          /* eigenpairs kept: inside the ellipse, residual <= res_tol */
    int32_t nbar;           /* rank chosen by the gap test */
    double gmax;            /* largest singular-value gap of the Hankel matrix */
    const rsrr_c128 *lam;   /* count eigenvalues, sorted by |lambda| then arg */
    const double *res;      /* count residuals ||T v||_2 / (sum_i |f_i| ||A_i||_1 ||v||_2) */
    const rsrr_c128 *V;     /* n x count eigenvectors, unit 2-norm columns */
} rsrr_result;

/* Fills `o` with the defaults listed above. */
void rsrr_opts_default(rsrr_opts *o);

/* Builds a handle: validates the descriptors, computes the sampling points and
 * the table f_i(z_j) on the host in FP64, copies the pattern and values to
 * the device, and allocates every device buffer of the handle (factors for
 * all N points, S, refinement work space).  The probe U is drawn from a
 * fixed seed; set it with rsrr_set_probe.  N >= 1, L >= 1.
 * Errors: EINVAL (bad descriptor), ENOMEM, ECUDA.  *out is NULL on error. */
rsrr_status rsrr_create(const rsrr_nep *nep, const rsrr_region *region, int32_t N,
                        int32_t L, const rsrr_opts *opts, rsrr_t **out);

/* Sets the probe matrix U (n x L, column major, Section 4.3 step 1).  U is
 * host memory if on_device == 0, else device memory; it is copied (async on
 * `stream` for device input, synchronous for host input). */
rsrr_status rsrr_set_probe(rsrr_t *h, const rsrr_c128 *U, int32_t on_device, void *stream);

/* Step 2: X_j = T(z_j)^{-1} U for all points, asynchronously on `stream`.
 * The outcome (ESINGULAR, ENOCONV) is known after the stream is synchronised
 * and is returned by rsrr_get_stats / rsrr_check. */
rsrr_status rsrr_sample(rsrr_t *h, void *stream);

/* Two-stage sampling (Section 5.4): appends `count` sampling points z_new
 * (host) to the handle -- typically the eigenvalues of a first rsrr_solve,
 * where the rational interpolation approach lets sampling points sit close to
 * eigenvalues -- and computes X_j = T(z_j)^{-1} U for the new points only,
 * with the same probe U and precision, asynchronously on `stream`.  The
 * samples of the earlier points stay resident and unchanged (bit for bit);
 * rsrr_project and rsrr_solve then use all N + count points.  The handle's
 * per-point buffers are reallocated for the larger N (the call waits for the
 * handle's earlier work first); rsrr_get_points, rsrr_get_samples and the
 * statistics report all points.  Requires a previous rsrr_sample.  Errors:
 * EINVAL (count < 1, a point not finite, f not finite there), ESTATE, ENOMEM,
 * ECUDA; the outcome of the new points' sampling is reported by rsrr_check. */
rsrr_status rsrr_add_points(rsrr_t *h, const rsrr_c128 *z_new, int32_t count, void *stream);

/* rsrr_sample for `count` band-path handles (sparse kind) of uneven sizes at
 * once, asynchronously on `stream`: each handle's assembly, then ONE
 * persistent grouped band LU over every sampling point of every handle (its
 * CTAs take (handle, point) tasks from a device queue, longest first; one
 * launch for the complex64 handles and one for the complex128 ones), then
 * each handle's solves and refinement.  The factors are bitwise those of the
 * one-CTA-per-point LU (RSRR_FLAG_ONE_CTA_LU), so each handle's samples are
 * those of its own rsrr_sample with that flag.  Check each handle's outcome
 * with rsrr_check.  The task table is allocated (cudaMallocAsync) and freed
 * on `stream`.  Errors: EINVAL (no handles, a dense handle, a handle twice),
 * ENOMEM, ECUDA (message in rsrr_last_error(NULL)) or a handle's own error. */
rsrr_status rsrr_sample_batch(rsrr_t *const *handles, int32_t count, void *stream);

/* Waits for `stream` and reports the outcome of the last rsrr_sample:
 * OK, ESINGULAR (a zero pivot; stats.singular_point names the point) or
 * ENOCONV (some column above eta_tol after max_refine sweeps). */
rsrr_status rsrr_check(rsrr_t *h, void *stream);

/* Steps 3-4, GPU part, on `stream`: column normalisation of S, orthonormal
 * basis Q (n x k) of its dominant singular subspace, and P_i = Q^H A_i Q.
 * Requires a previous rsrr_sample.  The call waits on `stream` twice (to size
 * the basis: the pivoted-Cholesky rank and the kept singular values); the
 * final products run asynchronously. */
rsrr_status rsrr_project(rsrr_t *h, void *stream);

/* Steps 4-5 (synchronises the handle's work first): SS-FULL on
 * T_Q(z) = sum_i f_i(z) P_i in FP64 -- the moments of T_Q^{-1} over the N_Q
 * quadrature nodes on the GPU (batched complex128 LU), the Hankel SVD and
 * the small eigenproblem on the host -- then v = Q g and residuals on the GPU.
 * Returns OK or WGAP (gap test failed; results still filled); ETIMEOUT if a
 * bounded wait of one of this handle's tensor-core product kernels ran out
 * since rsrr_sample (each handle counts its own in a device status word, so a
 * timeout in another handle or request never shows here).  After ETIMEOUT
 * the results of later calls on the same CUDA context are unverified: the
 * kernel that gave up stopped issuing work, but copies or MMAs it had issued
 * may not have finished within its bounded drain. */
rsrr_status rsrr_solve(rsrr_t *h, rsrr_result *out);

/* Copies S = [X_0 ... X_{N-1}] (n x N*L, column major, before normalisation)
 * into dst (device memory if dst_on_device, else host; async on stream for
 * device destinations, synchronous for host ones). */
rsrr_status rsrr_get_samples(rsrr_t *h, rsrr_c128 *dst, int32_t dst_on_device, void *stream);

/* Copies the per-column backward errors eta (N*L doubles, host) of the last
 * rsrr_sample.  Synchronises the handle's work. */
rsrr_status rsrr_get_eta(rsrr_t *h, double *dst);

/* Copies Q (n x k, column major) after rsrr_project; same memory rules as
 * rsrr_get_samples.  k is in rsrr_stats. */
rsrr_status rsrr_get_Q(rsrr_t *h, rsrr_c128 *dst, int32_t dst_on_device, void *stream);

/* Copies P_0 ... P_{m-1} (m consecutive k x k column-major blocks) after
 * rsrr_project; same memory rules as rsrr_get_samples.  For the Helmholtz
 * kind m is the number of Taylor terms (rsrr_stats.m): T_Q(z) =
 * sum_p (z - center)^p P_p. */
rsrr_status rsrr_get_projected(rsrr_t *h, rsrr_c128 *dst, int32_t dst_on_device, void *stream);

/* Copies the N sampling points (host). */
rsrr_status rsrr_get_points(rsrr_t *h, rsrr_c128 *dst);

/* Copies the result of the last rsrr_solve into caller-owned host buffers:
 * lam (count), res (count) and V (n x count, column major); any of them may
 * be NULL.  `capacity` is the number of eigenpairs the buffers hold; EINVAL
 * if it is below the count (the count is written to *count first, when
 * count is not NULL).  ESTATE before the first rsrr_solve. */
rsrr_status rsrr_copy_result(rsrr_t *h, int32_t capacity, int32_t *count, rsrr_c128 *lam,
                             double *res, rsrr_c128 *V);

/* Fills the statistics of the handle (synchronises the handle's work). */
rsrr_status rsrr_get_stats(rsrr_t *h, rsrr_stats *out);

/* One-line description of the last error on this handle ("" if none).  With
 * h == NULL: the last error of a failed rsrr_create or
 * rsrr_solve_band_noalloc on this thread. */
const char *rsrr_last_error(const rsrr_t *h);

/* Frees the handle and all its device memory.  NULL is allowed. */
void rsrr_destroy(rsrr_t *h);

/* Allocation-free solve of one banded system T X = U in complex128: the
 * factorisation (partial pivoting) and the triangular solves of rsrr_sample's
 * FP64 path, for a T the caller has already assembled.  The paper has no
 * counterpart; it exists for callers that cannot call cudaMalloc: plug-ins
 * whose host application's caching allocator or memory pool has reserved the
 * device memory up front, and latency-bound loops that must never enter the
 * allocator.  Nothing is allocated: the work space comes from a fixed 32 MiB
 * device array inside the library, which every GPU that loads the library
 * holds until the process exits.
 *   n, kl, ku  order and half-bandwidths of T (kl <= 480, kl and ku <= n - 1)
 *   band       device, (kl+ku+1) x n, LAPACK general band layout:
 *              T(i,j) at band[(ku + i - j) + j*(kl+ku+1)]
 *   L, U       device, n x L right-hand sides (column major); not modified
 *   X          device, n x L solution (column major); may not alias U
 *   stream     work is queued on it; the call waits for it before returning
 * Limit: 16*n*(2kl+ku+16) + 32*n*16 + 4*n bytes (each rounded up to 256) must
 * fit in 32 MiB, else RSRR_EINVAL with the needed size in the message; bands
 * whose solve would not fit in shared memory are refused the same way.  Every
 * check is made before anything is launched.
 * Returns OK, EINVAL, ESINGULAR (an exactly zero pivot) or ECUDA; the message
 * is in rsrr_last_error(NULL).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest
 * of the process; make that first call before any stream capture.  The entry
 * point does not survive a cudaDeviceReset.  Every call shares the one array
 * and overwrites all of it that it uses (no state carries over), so calls that
 * overlap on the GPU -- from several host threads or on several streams --
 * race: issue them one after another. */
rsrr_status rsrr_solve_band_noalloc(int64_t n, int32_t kl, int32_t ku, const rsrr_c128 *band,
                                    int32_t L, const rsrr_c128 *U, rsrr_c128 *X, void *stream);

/* One dense complex product C = alpha op(A) B + beta C on the device, by the
 * method the projection uses (Section 4.3's Gram matrices and Q^H A_i Q are
 * such products); exposed so that callers and tests can use or check it alone.
 *   M, N, K    op(A) is M x K, B is K x N, C is M x N
 *   conjA      0: op(A) = A (M x K),  1: op(A) = A^H (A is K x M)
 *   A, B, C    device, column major with leading dimensions lda, ldb, ldc;
 *              C may not alias A or B
 *   alpha, beta  real scalars; beta = 0 ignores the contents of C
 *   method     RSRR_GEMM_FP64, RSRR_GEMM_OZAKI or RSRR_GEMM_AUTO
 *   hermitian  nonzero with conjA, A == B, lda == ldb, M == N: the result is
 *              Hermitian; only its upper block triangle is computed and the
 *              rest mirrored (beta must be 0)
 *   max_ws_bytes  0: work space for the whole product; else its upper bound
 *              (the product then runs in chunks of K)
 *   stream     work is queued on it; the call waits for it before returning
 * Work space is allocated and freed inside the call.  Returns OK, EINVAL,
 * ENOMEM (work space), ETIMEOUT (a bounded wait of the tensor-core kernel ran
 * out) or ECUDA; the message is in rsrr_last_error(NULL). */
rsrr_status rsrr_zgemm(int32_t M, int32_t N, int32_t K, int32_t conjA, const rsrr_c128 *A,
                       int64_t lda, const rsrr_c128 *B, int64_t ldb, rsrr_c128 *C, int64_t ldc,
                       double alpha, double beta, int32_t method, int32_t hermitian,
                       size_t max_ws_bytes, void *stream);

/* Failure detection without a GPU fault: one thread waits, with the bounded
 * mbarrier wait of the tensor-core product kernel, on a barrier that nothing
 * completes, giving up after `tries` polls (1 .. 2^20).  The wait is counted
 * in a status word of this call (allocated and freed inside it), the same way
 * a wait of a product kernel is counted in its caller's word: rsrr_zgemm's
 * own, or the handle's for rsrr_sample / rsrr_project (read by rsrr_solve).
 * Returns ETIMEOUT when the wait ran out and was counted, with the CUDA
 * context still usable; OK (with a message) if it was not counted; EINVAL or
 * ECUDA otherwise.  Waits for `stream` before and after. */
rsrr_status rsrr_check_wait_timeout(int32_t tries, void *stream);

/* Host-only view of what rsrr_create prepares, without touching the GPU:
 * the N sampling points z_j (step 1; Section 5.1 trapezoid nodes on the
 * ellipse, or the explicit points), the coefficient table f_i(z_j) (sparse
 * kind: N x m, point-major, coef[j * m + i]; not written for the Helmholtz
 * kind) and the half-bandwidths kl, ku detected from the pattern (0 for the
 * Helmholtz kind).  Outputs are host memory owned by the caller; any of them
 * may be NULL.  Same arguments, validation and errors as rsrr_create. */
rsrr_status rsrr_describe(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                          const rsrr_opts *opts, rsrr_c128 *z, rsrr_c128 *coef, int32_t *kl,
                          int32_t *ku);

/* Device bytes a handle for this problem holds at its peak (its buffers, the
 * projection work space and rsrr_solve's temporaries), without allocating
 * anything or touching the GPU.  Same arguments and validation as
 * rsrr_create; the request server admits requests by this number. */
rsrr_status rsrr_estimate_bytes(const rsrr_nep *nep, const rsrr_region *region, int32_t N,
                                int32_t L, const rsrr_opts *opts, size_t *bytes);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of whole RSRR solves on one GPU.
 *
 * Requests (a NEP, a region, N, L, options and optionally a probe U) are
 * queued by rsrr_server_submit and run by `slots` worker threads, each with
 * its own non-blocking CUDA stream: a request is admitted, in arrival order,
 * as soon as a slot is free and its rsrr_estimate_bytes fit in what the
 * memory budget has left (a later request may pass a waiting one that does
 * not fit yet, at most 8 times).  Admitted requests allocate from the
 * server's stream-ordered memory pool and run rsrr_sample, rsrr_project and
 * rsrr_solve; their kernels overlap on the device with those of the other
 * admitted requests, and each request's host work overlaps with the others'
 * GPU work.  Results (eigenvalues, residuals, eigenvectors) are copied to
 * host memory owned by the server.  Each request runs the same kernels on
 * the same inputs as a lone handle would: its results do not depend on what
 * else runs.
 * ------------------------------------------------------------------------ */
typedef struct rsrr_server rsrr_server_t;

typedef struct {
    int32_t slots;            /* requests on the device at once, 1..64, default 4 */
    int32_t keep;             /* nonzero: a finished request keeps its handle (factors,
                                 S, Q, P_i) resident, and its bytes counted against
                                 the budget, until rsrr_server_release; default 0 */
    int64_t mem_budget_bytes; /* device bytes the admitted requests may hold together,
                                 default 150e9 */
    int32_t device;           /* CUDA device; -1 (default): the current device */
    int32_t reserved;
} rsrr_server_opts;

typedef struct {
    int64_t id;
    int32_t status;        /* the request's outcome: OK, WGAP (results filled) or an error */
    int32_t count, nbar, k, refine_sweeps;
    double gmax, max_eta;
    double t_submit;       /* seconds since rsrr_server_create: submission (arrival), */
    double t_admit;        /* admission (slot and memory granted) and */
    double t_done;         /* results on the host */
    double t_sample;       /* wall seconds of the request's rsrr_sample (to its outcome), */
    double t_project;      /* rsrr_project (to its last product) and */
    double t_solve;        /* rsrr_solve (SS-FULL, eigenvectors, residuals) */
    size_t device_bytes;   /* bytes admitted against the budget */
    int64_t n;
    const rsrr_c128 *lam;  /* count eigenvalues, as rsrr_result */
    const double *res;     /* count residuals, as rsrr_result */
    const rsrr_c128 *V;    /* n x count eigenvectors, as rsrr_result */
    const char *error;     /* one line if status < 0, else "" */
} rsrr_reply;

typedef struct {
    int64_t submitted, completed, failed;
    int32_t queued, active, peak_active, reserved;
    size_t used_bytes, peak_bytes, budget_bytes;
    double now;            /* seconds since rsrr_server_create */
} rsrr_server_stats;

/* Fills `o` with the defaults listed above. */
void rsrr_server_opts_default(rsrr_server_opts *o);

/* Starts a server on the device (memory pool, worker threads and streams).
 * Errors: EINVAL (slots or budget out of range), ECUDA, ENOMEM; message in
 * rsrr_last_error(NULL). */
rsrr_status rsrr_server_create(const rsrr_server_opts *opts, rsrr_server_t **out);

/* Queues one request and returns its id (> 0).  The descriptors are
 * validated and copied as by rsrr_create, and U (host, n x L, column major,
 * NULL for the default probe) is copied; the caller may free all of them on
 * return.  opts.host_threads == 0 gives the request's host work
 * cores / slots threads.  Errors: EINVAL (descriptor), ENOMEM (the request
 * alone exceeds the budget), ESTATE (server shutting down). */
rsrr_status rsrr_server_submit(rsrr_server_t *server, const rsrr_nep *nep,
                               const rsrr_region *region, int32_t N, int32_t L,
                               const rsrr_opts *opts, const rsrr_c128 *U, int64_t *id);

/* Waits up to timeout_s seconds (< 0: no limit) for request `id` and fills
 * *out; the arrays it points to stay valid until rsrr_server_release(id).
 * Returns OK (the request's own outcome is out->status), ETIMEOUT (not
 * finished in time; *out untouched) or EINVAL (unknown id). */
rsrr_status rsrr_server_wait(rsrr_server_t *server, int64_t id, double timeout_s,
                             rsrr_reply *out);

/* With opts.keep: the finished request's handle, for rsrr_get_Q,
 * rsrr_get_projected, rsrr_get_samples, rsrr_get_stats ...; owned by the
 * server (do not destroy it).  NULL if the request is unknown, unfinished,
 * failed, or the server does not keep handles. */
rsrr_t *rsrr_server_handle(rsrr_server_t *server, int64_t id);

/* Forgets a finished request: frees its host results and, with keep, its
 * handle, whose bytes go back to the budget.  EINVAL (unknown id), ESTATE
 * (not finished). */
rsrr_status rsrr_server_release(rsrr_server_t *server, int64_t id);

/* Counters and memory use of the server. */
rsrr_status rsrr_server_get_stats(rsrr_server_t *server, rsrr_server_stats *out);

/* Lets the admitted requests finish, drops the queued ones, frees every
 * request, the pool and the workers.  NULL is allowed. */
void rsrr_server_destroy(rsrr_server_t *server);

#ifdef __cplusplus
}
#endif

#endif /* RSRR_H */
