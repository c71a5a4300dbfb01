// Host side of the C ABI declared in include/rsrr.h: descriptor validation,
// sampling points and coefficient table (RSRR step 1, Section 4.3), device
// buffers, and the orchestration of the sampling kernels (step 2).
#include <algorithm>
#include <limits>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rsrr.h"
#include "rsrr_handle.h"

using cplx = std::complex<double>;

namespace rsrr {

// last error of a call without a handle (rsrr_create, rsrr_solve_band_noalloc)
std::string &thread_error() {
    thread_local std::string s;
    return s;
}

cplx eval_fn_host(const rsrr_fn &f, cplx z) {
    cplx base;
    switch (f.kind) {
        case RSRR_F_ONE: base = 1.0; break;
        case RSRR_F_ZPOW: {
            base = 1.0;
            const int p = (int)f.param;
            for (int q = 0; q < p; ++q) base *= z;
            break;
        }
        case RSRR_F_RATIONAL: base = z / (z - f.param); break;
        case RSRR_F_INV: base = 1.0 / (f.param - z); break;
        case RSRR_F_SQRT: base = std::sqrt(z * z - f.param * f.param); break;
        case RSRR_F_EXP: base = std::exp(-f.param * z); break;
        case RSRR_F_TAYLOR: {
            base = 1.0;
            const cplx d = z - cplx(f.shift.re, f.shift.im);
            for (int q = 0; q < f.power; ++q) base *= d;
            break;
        }
        default: base = cplx(NAN, NAN);  // callbacks are evaluated by Handle::eval_terms
    }
    return cplx(f.scale.re, f.scale.im) * base;
}

// complex normal entries (g1 + i g2)/sqrt(2) from splitmix64 + Box-Muller;
// seed 0 is the library's historical default stream
void default_probe(std::vector<double2> &U, size_t count, uint64_t seed) {
    U.resize(count);
    uint64_t st = 0x9E3779B97F4A7C15ull + seed * 0xD1B54A32D192ED03ull;
    auto next = [&st]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (size_t q = 0; q < count; ++q) {
        const double r = std::sqrt(-2.0 * std::log(next())), t = 2.0 * M_PI * next();
        U[q] = make_double2(r * std::cos(t) / std::sqrt(2.0), r * std::sin(t) / std::sqrt(2.0));
    }
}

rsrr_status Handle::eval_terms(const cplx *zz, int64_t count, std::vector<cplx> &out) {
    const int mt = (int)fn.size();
    out.assign((size_t)count * mt, cplx(0.0, 0.0));
    std::vector<rsrr_c128> zin, val;
    for (int t = 0; t < mt; ++t) {
        const rsrr_fn &f = fn[t];
        if (f.kind == RSRR_F_CALLBACK) {
            if (!cb) return fail(RSRR_EINVAL, "callback term without a callback");
            if (zin.empty()) {
                zin.resize(count);
                for (int64_t q = 0; q < count; ++q) zin[q] = rsrr_c128{zz[q].real(), zz[q].imag()};
            }
            val.assign(count, rsrr_c128{NAN, NAN});
            cb(fn_src[t], zin.data(), count, val.data(), cb_user);
            const cplx sc(f.scale.re, f.scale.im);
            for (int64_t q = 0; q < count; ++q) out[(size_t)q * mt + t] = sc * cplx(val[q].re, val[q].im);
        } else {
            for (int64_t q = 0; q < count; ++q) out[(size_t)q * mt + t] = eval_fn_host(f, zz[q]);
        }
    }
    for (const cplx &v : out)
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
            return fail(RSRR_EINVAL, "f_i is not finite at a point where it is needed");
    return RSRR_OK;
}

// Gauss-Legendre nodes (ascending) and weights of the n-point rule on [-1, 1]:
// Newton's method on the Legendre polynomial P_n from the three-term
// recurrence (k + 1) P_{k+1} = (2k + 1) x P_k - k P_{k-1}, started at the
// asymptotic root estimates cos(pi (i + 3/4) / (n + 1/2)); with
// P_n' = n (x P_n - P_{n-1}) / (x^2 - 1), the weights are
// 2 / ((1 - x^2) P_n'(x)^2).
static void legendre_at(int n, double t, double &pn, double &dpn) {
    double p0 = 1.0, p1 = t;
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    pn = p1;
    dpn = n * (t * p1 - p0) / (t * t - 1.0);
}

static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pn = 0.0, dpn = 1.0;
        for (int it = 0; it < 100; ++it) {
            legendre_at(n, t, pn, dpn);
            const double dt = pn / dpn;
            t -= dt;
            if (std::fabs(dt) <= 1e-15 * std::fabs(t) + 1e-300) break;
        }
        legendre_at(n, t, pn, dpn);
        const double wt = 2.0 / ((1.0 - t * t) * dpn * dpn);
        x[n - 1 - i] = t;
        x[i] = -t;
        w[i] = w[n - 1 - i] = wt;
    }
    if (n & 1) x[n / 2] = 0.0;
}

// the rectangle's vertices counterclockwise from center - a - i b (v[4] = v[0])
static void rect_vertices(const rsrr_region &r, cplx v[5]) {
    const cplx c(r.center.re, r.center.im);
    v[0] = c + cplx(-r.a, -r.b);
    v[1] = c + cplx(r.a, -r.b);
    v[2] = c + cplx(r.a, r.b);
    v[3] = c + cplx(-r.a, r.b);
    v[4] = v[0];
}

// Gauss-Legendre nodes on the rectangle's sides (count[s] on side s, along
// its direction) and the contour weights dz/(2 pi) = (q - p) w / (4 pi)
static void rect_rule(const rsrr_region &r, const int count[4], std::vector<cplx> &z, std::vector<cplx> *wz) {
    cplx v[5];
    rect_vertices(r, v);
    z.clear();
    if (wz) wz->clear();
    std::vector<double> x, w;
    for (int sd = 0; sd < 4; ++sd) {
        gauss_legendre(count[sd], x, w);
        const cplx p = v[sd], q = v[sd + 1];
        for (int k = 0; k < count[sd]; ++k) {
            z.push_back(0.5 * (p + q) + 0.5 * (q - p) * x[k]);
            if (wz) wz->push_back(0.5 * (q - p) * w[k] / (2.0 * M_PI));
        }
    }
}

void Handle::contour_quadrature(int NQ, std::vector<cplx> &zq, std::vector<cplx> &wq) const {
    zq.clear();
    wq.clear();
    const cplx gamma(region.center.re, region.center.im);
    if (region.kind != RSRR_REGION_RECT) {
        for (int q = 0; q < NQ; ++q) {
            const double t = 2.0 * M_PI * (q + 0.5) / NQ;
            zq.push_back(gamma + cplx(region.a * std::cos(t), region.b * std::sin(t)));
            wq.push_back(cplx(-region.a * std::sin(t), region.b * std::cos(t)) / (double)NQ);
        }
        return;
    }
    // composite Gauss: side s in max(1, round(NQ len_s / (10 perimeter))) equal
    // panels with the 10-point rule each
    constexpr int PANEL = 10;
    std::vector<double> x, w;
    gauss_legendre(PANEL, x, w);
    cplx v[5];
    rect_vertices(region, v);
    const double per = 4.0 * (region.a + region.b);
    for (int sd = 0; sd < 4; ++sd) {
        const cplx p = v[sd], q = v[sd + 1];
        const int P = std::max(1, (int)std::lround(NQ * std::abs(q - p) / (PANEL * per)));
        for (int t = 0; t < P; ++t) {
            const cplx a0 = p + (q - p) * ((double)t / P), a1 = p + (q - p) * ((double)(t + 1) / P);
            for (int k = 0; k < PANEL; ++k) {
                zq.push_back(0.5 * (a0 + a1) + 0.5 * (a1 - a0) * x[k]);
                wq.push_back(0.5 * (a1 - a0) * w[k] / (2.0 * M_PI));
            }
        }
    }
}

bool Handle::inside(cplx lam) const {
    const double x = (lam.real() - region.center.re) / region.a;
    const double y = (lam.imag() - region.center.im) / region.b;
    if (region.kind == RSRR_REGION_RECT) return std::fabs(x) < 1.0 && std::fabs(y) < 1.0;
    return x * x + y * y < 1.0;
}

// weights w_i of the moment methods (up to a common factor): trapezoid
// weights (1/N) phi'(alpha_i) on the ellipse (Eq. 58), Chebyshev weights
// (-1)^i sin((2i + 1) pi / 2N) on an interval (Eq. 43), the contour weights
// dz/(2 pi) at Gauss-Legendre nodes on a rectangle (Section 5.4), otherwise the
// barycentric weights 1 / prod_{j != i} (z_i - z_j) (Eq. 19) with every factor
// scaled by 2 / rho and formed through logarithms
void Handle::moment_weights(std::vector<cplx> &w) const {
    const int n_ = (int)z.size();
    w.assign(n_, cplx(0.0, 0.0));
    const double rho = std::max(region.a, region.b);
    const cplx gamma(region.center.re, region.center.im);
    if (region.kind == RSRR_REGION_ELLIPSE && !points_added) {
        for (int j = 0; j < n_; ++j) {
            const double al = 2.0 * M_PI * (j + 0.5) / n_;
            w[j] = cplx(-region.a * std::sin(al), region.b * std::cos(al)) / (double)n_;
        }
        return;
    }
    if (region.kind == RSRR_REGION_INTERVAL && !points_added) {
        for (int j = 0; j < n_; ++j)
            w[j] = cplx(((j & 1) ? -1.0 : 1.0) * std::sin((2.0 * j + 1.0) * M_PI / (2.0 * n_)), 0.0);
        return;
    }
    if (rect_gl && !points_added) {  // Gauss-Legendre nodes: the contour weights dz / (2 pi)
        const int ny = n_ / 2 - region.nx;
        const int cnt[4] = {region.nx, ny, region.nx, ny};
        std::vector<cplx> zz;
        rect_rule(region, cnt, zz, &w);
        return;
    }
    std::vector<cplx> lw(n_);
    double top = -1e300;
    for (int i = 0; i < n_; ++i) {
        cplx acc = 0.0;
        for (int j = 0; j < n_; ++j)
            if (j != i) acc -= std::log((z[i] - z[j]) * (2.0 / rho));
        lw[i] = acc;
        top = std::max(top, acc.real());
    }
    for (int i = 0; i < n_; ++i) w[i] = std::exp(lw[i] - top);
    (void)gamma;
}

double Handle::residual_scale(const cplx *f_held) const {
    double scale = 0.0;
    for (size_t t = 0; t < fn.size(); ++t)
        if (!fn_imag[t]) scale += std::abs(f_held[t]) * a1[fn_src[t]];  // |i f_u| = |f_u|: count once
    return scale;
}

rsrr_status Handle::fail(rsrr_status st, const char *what, cudaError_t e) {
    char buf[512];
    if (e != cudaSuccess)
        snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof buf, "%s", what);
    err = buf;
    return st;
}

template <typename T> cudaError_t Handle::alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return raw_alloc((void **)p, sizeof(T) * count);
}

// device memory owned by the handle: cudaMalloc, or the server's
// stream-ordered pool on hs; in dry mode only the bytes are counted
cudaError_t Handle::raw_alloc(void **p, size_t bytes) {
    *p = nullptr;
    if (dry) {
        device_bytes += bytes;
        return cudaSuccess;
    }
    cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, hs) : cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        allocations.push_back(*p);
        device_bytes += bytes;
    }
    return e;
}

// frees a buffer obtained outside alloc() (temporary buffers of rsrr_solve)
cudaError_t Handle::raw_free(void *p) { return pool ? cudaFreeAsync(p, hs) : cudaFree(p); }

// waits for the handle's work: its own stream, or the whole device
cudaError_t Handle::wait() { return hs ? cudaStreamSynchronize(hs) : cudaDeviceSynchronize(); }

Handle::~Handle() {
    drop_graph();
    for (void *p : allocations) {
        if (pool) cudaFreeAsync(p, hs);
        else cudaFree(p);
    }
    for (auto &e : events)
        if (e) cudaEventDestroy(e);
}

cudaError_t EventPool::next(cudaEvent_t *out) {
    if (used == (int)ev.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        ev.push_back(e);
    }
    *out = ev[used++];
    return cudaSuccess;
}

cudaError_t EventPool::sum_pairs_ms(double *ms) const {
    double tot = 0.0;
    for (int i = 0; i + 1 < used; i += 2) {
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
        if (e != cudaSuccess) return e;
        tot += t;
    }
    *ms = tot;
    return cudaSuccess;
}

EventPool::~EventPool() {
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
}

// next event of the GEMM timing pool
cudaError_t Handle::gemm_event(cudaEvent_t *out) { return gemm_pool.next(out); }

}  // namespace rsrr

using rsrr::Handle;

#define CK(expr, what)                                                   \
    do {                                                                 \
        cudaError_t _e = (expr);                                         \
        if (_e != cudaSuccess) return h->fail(RSRR_ECUDA, what, _e);     \
    } while (0)

extern "C" {

void rsrr_opts_default(rsrr_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = RSRR_PREC_MIXED;
    o->max_refine = 8;
    o->eta_tol = 1e-10;
    o->delta = 1e-14;
    o->delta_floor = 0.0;  // automatic: 0.1 eta_tol (mixed), 1e-12 (FP64)
    o->tol_gap = 1e3;
    o->res_tol = 1e-6;
    o->NQ = 500;
    o->KQ = 2;
    o->host_threads = 0;
    o->gemm = RSRR_GEMM_AUTO;
    o->method = RSRR_METHOD_RSRR;
    o->K = 2;
    o->refine = RSRR_REFINE_IR;
    o->gmres_m = 4;
    o->chunk_points = 0;
    o->reserved = 0;
}

static rsrr_status create_fail(const char *msg) {
    rsrr::thread_error() = msg;
    return RSRR_EINVAL;
}

namespace rsrr {
rsrr_status prepare_dense(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                          const rsrr_opts *opts, Handle **out);
}

rsrr_status rsrr_create(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                        const rsrr_opts *opts, rsrr_t **out) {
    if (!out) return create_fail("rsrr_create: out is NULL");
    *out = nullptr;
    Handle *h = nullptr;
    rsrr_status st = rsrr::prepare(nep, region, N, L, opts, &h);
    if (st != RSRR_OK) return st;
    if (h->opts.mem_budget_bytes > 0) {
        size_t need = h->estimate_bytes();
        const size_t budget = (size_t)h->opts.mem_budget_bytes;
        if (need > budget && (h->opts.flags & RSRR_FLAG_CHUNK_POINTS) && !h->dense && h->N > 1) {
            // the band storage of as many points as fit: need(f) is affine in f
            h->fcap = 1;
            const size_t need1 = h->estimate_bytes();
            h->fcap = 2;
            const size_t per = h->estimate_bytes() - need1;
            h->fcap = 1;
            if (need1 <= budget && per > 0)
                h->fcap = (int)std::min<size_t>((size_t)h->N, 1 + (budget - need1) / per);
            while (h->fcap > 1 && h->estimate_bytes() > budget) --h->fcap;
            need = h->estimate_bytes();
        }
        if (need > budget) {
            char buf[160];
            snprintf(buf, sizeof buf, "rsrr_create: the handle needs %zu device bytes, mem_budget_bytes is %lld",
                     need, (long long)h->opts.mem_budget_bytes);
            rsrr::thread_error() = buf;
            delete h;
            return RSRR_ENOMEM;
        }
    }
    st = h->allocate();
    if (st != RSRR_OK) {
        rsrr::thread_error() = h->err;
        delete h;
        return st;
    }
    *out = reinterpret_cast<rsrr_t *>(h);
    return RSRR_OK;
}

rsrr_status rsrr_estimate_bytes(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                                const rsrr_opts *opts, size_t *bytes) {
    if (!bytes) return create_fail("rsrr_estimate_bytes: bytes is NULL");
    *bytes = 0;
    Handle *h = nullptr;
    rsrr_status st = rsrr::prepare(nep, region, N, L, opts, &h);
    if (st != RSRR_OK) return st;
    *bytes = h->estimate_bytes();
    delete h;
    return RSRR_OK;
}

rsrr_status rsrr_describe(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                          const rsrr_opts *opts, rsrr_c128 *z, rsrr_c128 *coef, int32_t *kl,
                          int32_t *ku) {
    Handle *h = nullptr;
    rsrr_status st = rsrr::prepare(nep, region, N, L, opts, &h);
    if (st != RSRR_OK) return st;
    if (z)
        for (int j = 0; j < h->N; ++j) z[j] = rsrr_c128{h->z[j].real(), h->z[j].imag()};
    if (coef && (!h->dense || h->dense_terms))
        for (size_t e = 0; e < h->h_coef.size(); ++e) coef[e] = rsrr_c128{h->h_coef[e].x, h->h_coef[e].y};
    if (kl) *kl = h->dense ? 0 : h->kl;
    if (ku) *ku = h->dense ? 0 : h->ku;
    delete h;
    return RSRR_OK;
}

}  // extern "C"

namespace rsrr {

static rsrr_status check_fns(const rsrr_nep *nep) {
    for (int i = 0; i < nep->m; ++i) {
        const rsrr_fn &f = nep->fn[i];
        if (f.kind < RSRR_F_ONE || f.kind > RSRR_F_CALLBACK) return create_fail("rsrr_create: bad fn kind");
        if (f.kind == RSRR_F_ZPOW && (f.param < 0 || f.param != std::floor(f.param) || f.param > 64))
            return create_fail("rsrr_create: ZPOW needs a small non-negative integer");
        if (f.kind == RSRR_F_TAYLOR && (f.power < 0 || f.power > 64))
            return create_fail("rsrr_create: TAYLOR power out of range (0 .. 64)");
        if (f.kind == RSRR_F_CALLBACK && !nep->callback)
            return create_fail("rsrr_create: CALLBACK term without nep->callback");
    }
    return RSRR_OK;
}

static rsrr_status check_common(const rsrr_region *region, const rsrr_opts *opts, int N) {
    if (!(region->a > 0.0) || !(region->b > 0.0))
        return create_fail("rsrr_create: ellipse semi-axes must be > 0");
    if (region->kind != RSRR_REGION_ELLIPSE && region->kind != RSRR_REGION_POINTS &&
        region->kind != RSRR_REGION_INTERVAL && region->kind != RSRR_REGION_RECT)
        return create_fail("rsrr_create: unknown region kind");
    if (region->kind == RSRR_REGION_POINTS && !region->points)
        return create_fail("rsrr_create: points region without points");
    if (region->kind == RSRR_REGION_RECT && !region->points &&
        (N < 4 || (N & 1) || region->nx < 1 || region->nx > N / 2 - 1))
        return create_fail("rsrr_create: a rectangle needs N even and 1 <= nx <= N/2 - 1");
    const int prec = opts ? opts->precision : RSRR_PREC_MIXED;
    if (prec != RSRR_PREC_FP64 && prec != RSRR_PREC_MIXED)
        return create_fail("rsrr_create: unknown precision");
    if (opts && (opts->gemm < RSRR_GEMM_AUTO || opts->gemm > RSRR_GEMM_OZAKI_MMA))
        return create_fail("rsrr_create: unknown gemm method");
    if (opts && opts->mem_budget_bytes < 0) return create_fail("rsrr_create: negative mem_budget_bytes");
    if (opts && (opts->method < RSRR_METHOD_RSRR || opts->method > RSRR_METHOD_SS_RI))
        return create_fail("rsrr_create: unknown method");
    if (opts && opts->method != RSRR_METHOD_RSRR && (opts->K < 1 || opts->K > N))
        return create_fail("rsrr_create: the moment methods need 1 <= K <= N");
    if (opts && (opts->refine < RSRR_REFINE_IR || opts->refine > RSRR_REFINE_GMRES))
        return create_fail("rsrr_create: unknown refinement");
    if (opts && opts->refine == RSRR_REFINE_GMRES && (opts->gmres_m < 1 || opts->gmres_m > 16))
        return create_fail("rsrr_create: gmres_m out of range (1 .. 16)");
    if (opts && opts->chunk_points < 0) return create_fail("rsrr_create: negative chunk_points");
    return RSRR_OK;
}

// step 1: the sampling points, trapezoid nodes on the ellipse (Eq. 58,
// Section 5.1), the explicit points (any points, Section 3.3), the
// Chebyshev points of the first kind on the major axis (Eq. 42) or
// Gauss-Legendre nodes on the sides of a rectangle (Section 5.4)
static void fill_points(Handle *h, const rsrr_region *region, int N) {
    if (region->kind == RSRR_REGION_RECT && !region->points) {
        const int ny = N / 2 - region->nx;
        const int cnt[4] = {region->nx, ny, region->nx, ny};
        rect_rule(*region, cnt, h->z, nullptr);
        h->rect_gl = true;
        return;
    }
    h->z.resize(N);
    for (int j = 0; j < N; ++j) {
        if (region->kind == RSRR_REGION_POINTS || region->kind == RSRR_REGION_RECT) {
            h->z[j] = cplx(region->points[j].re, region->points[j].im);
        } else if (region->kind == RSRR_REGION_INTERVAL) {
            h->z[j] = cplx(region->center.re + region->a * std::cos((2.0 * j + 1.0) * M_PI / (2.0 * N)),
                           region->center.im);
        } else {
            const double al = 2.0 * M_PI * (j + 0.5) / N;
            h->z[j] = cplx(region->center.re + region->a * std::cos(al),
                           region->center.im + region->b * std::sin(al));
        }
    }
}

// the coefficient table f_i(z_j) of the held terms, N x m point-major
static rsrr_status fill_coef(Handle *h) {
    std::vector<cplx> f;
    rsrr_status st = h->eval_terms(h->z.data(), h->N, f);
    if (st != RSRR_OK) {
        thread_error() = "rsrr_create: " + h->err;
        return st;
    }
    h->h_coef.resize(f.size());
    for (size_t e = 0; e < f.size(); ++e) h->h_coef[e] = make_double2(f[e].real(), f[e].imag());
    return RSRR_OK;
}

static Handle *new_handle(const rsrr_nep *nep, const rsrr_region *region, int N, int L,
                          const rsrr_opts *opts) {
    Handle *h = new (std::nothrow) Handle();
    if (!h) return nullptr;
    if (opts) h->opts = *opts; else rsrr_opts_default(&h->opts);
    h->seed = h->opts.seed;
    h->n = nep->n;
    h->N = N;
    h->fcap = N;
    if (nep->kind == RSRR_NEP_SPARSE && h->opts.chunk_points > 0) h->fcap = std::min(N, h->opts.chunk_points);
    h->L = L;
    h->region = *region;
    h->region.points = nullptr;
    h->cb = nep->callback;
    h->cb_user = nep->callback_user;
    return h;
}

rsrr_status prepare_dense(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                          const rsrr_opts *opts, Handle **out);
rsrr_status prepare_dense_terms(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                                const rsrr_opts *opts, Handle **out);

rsrr_status prepare(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                    const rsrr_opts *opts, Handle **out) {
    *out = nullptr;
    rsrr::thread_error().clear();
    if (!nep || !region) return create_fail("rsrr_create: nep or region is NULL");
    if (nep->n < 1 || nep->n > (int64_t)1 << 30) return create_fail("rsrr_create: n out of range");
    if (N < 1 || L < 1) return create_fail("rsrr_create: N and L must be >= 1");
    if (nep->kind != RSRR_NEP_SPARSE && nep->kind != RSRR_NEP_HELMHOLTZ && nep->kind != RSRR_NEP_DENSE)
        return create_fail("rsrr_create: unknown NEP kind");
    rsrr_status cst = check_common(region, opts, N);
    if (cst != RSRR_OK) return cst;
    if (opts && (opts->flags & RSRR_FLAG_REAL) && nep->kind != RSRR_NEP_SPARSE)
        return create_fail("rsrr_create: RSRR_FLAG_REAL needs the sparse kind");
    if (nep->kind == RSRR_NEP_HELMHOLTZ) return rsrr::prepare_dense(nep, region, N, L, opts, out);
    if (nep->m < 1 || nep->m > RSRR_MAX_TERMS) return create_fail("rsrr_create: m out of range");
    if ((cst = check_fns(nep)) != RSRR_OK) return cst;
    if (nep->kind == RSRR_NEP_DENSE) return rsrr::prepare_dense_terms(nep, region, N, L, opts, out);
    if (!nep->row_ptr || !nep->col_idx || !nep->values)
        return create_fail("rsrr_create: pattern or values NULL");
    const int64_t n = nep->n;
    const int64_t nnz = nep->row_ptr[n];
    if (nep->row_ptr[0] != 0 || nnz < 1 || nnz > INT32_MAX)
        return create_fail("rsrr_create: bad row_ptr");
    // pattern checks and bandwidths
    int64_t kl = 0, ku = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (nep->row_ptr[i + 1] < nep->row_ptr[i]) return create_fail("rsrr_create: row_ptr decreasing");
        for (int64_t e = nep->row_ptr[i]; e < nep->row_ptr[i + 1]; ++e) {
            const int64_t c = nep->col_idx[e];
            if (c < 0 || c >= n) return create_fail("rsrr_create: column index out of range");
            kl = std::max(kl, i - c);
            ku = std::max(ku, c - i);
        }
    }
    if (kl > rsrr::KL_MAX) return create_fail("rsrr_create: lower bandwidth above 480");
    const int prec = opts ? opts->precision : RSRR_PREC_MIXED;

    Handle *h = new_handle(nep, region, N, L, opts);
    if (!h) { rsrr::thread_error() = "rsrr_create: out of host memory"; return RSRR_ENOMEM; }
    h->nnz = nnz;
    h->kl = (int)kl; h->ku = (int)ku;
    h->geom.kl = (int)kl;
    h->geom.ku = (int)ku;
    h->geom.nb = prec == RSRR_PREC_MIXED ? rsrr::NB_C64 : rsrr::NB_C128;
    h->geom.ldab = 2 * (int)kl + (int)ku + h->geom.nb;

    // host copies of the pattern (int32 row pointers; nnz < 2^31 checked)
    h->h_row_ptr.resize(n + 1);
    for (int64_t i = 0; i <= n; ++i) h->h_row_ptr[i] = (int32_t)nep->row_ptr[i];
    h->h_col_idx.assign(nep->col_idx, nep->col_idx + nnz);
    // the terms as held: real values one term each; complex values Re A_u with
    // f_u and, unless every imaginary part is zero, Im A_u with i f_u
    // (T = sum_u f_u (Re A_u + i Im A_u) exactly); ||A_u||_1 of every caller term
    h->a1.assign(nep->m, 0.0);
    for (int u = 0; u < nep->m; ++u) {
        std::vector<double> colsum(n, 0.0);
        if (nep->values_complex) {
            const double *v = nep->values + (size_t)2 * u * nnz;
            bool imag = false;
            for (int64_t e = 0; e < nnz; ++e) {
                colsum[h->h_col_idx[e]] += std::hypot(v[2 * e], v[2 * e + 1]);
                imag = imag || v[2 * e + 1] != 0.0;
            }
            for (int64_t e = 0; e < nnz; ++e) h->h_vals.push_back(v[2 * e]);
            h->fn.push_back(nep->fn[u]);
            h->fn_src.push_back(u);
            h->fn_imag.push_back(0);
            if (imag) {
                for (int64_t e = 0; e < nnz; ++e) h->h_vals.push_back(v[2 * e + 1]);
                rsrr_fn fi = nep->fn[u];
                fi.scale = rsrr_c128{-nep->fn[u].scale.im, nep->fn[u].scale.re};  // i * scale
                h->fn.push_back(fi);
                h->fn_src.push_back(u);
                h->fn_imag.push_back(1);
            }
        } else {
            const double *v = nep->values + (size_t)u * nnz;
            for (int64_t e = 0; e < nnz; ++e) colsum[h->h_col_idx[e]] += std::fabs(v[e]);
            h->h_vals.insert(h->h_vals.end(), v, v + nnz);
            h->fn.push_back(nep->fn[u]);
            h->fn_src.push_back(u);
            h->fn_imag.push_back(0);
        }
        for (double c : colsum) h->a1[u] = std::max(h->a1[u], c);
    }
    for (double v : h->h_vals)
        if (!std::isfinite(v)) {
            delete h;
            return create_fail("rsrr_create: values must be finite");
        }
    h->m = (int)h->fn.size();
    // duplicates inside a row are rejected (a CSC lookup needs unique entries)
    {
        std::vector<int32_t> cnt(n + 1, 0);
        for (int64_t e = 0; e < nnz; ++e) cnt[h->h_col_idx[e] + 1]++;
        std::vector<int32_t> cptr(n + 1, 0);
        for (int64_t c = 0; c < n; ++c) cptr[c + 1] = cptr[c] + cnt[c + 1];
        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
        std::vector<int32_t> crow(nnz), cperm(nnz);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = h->h_row_ptr[i]; e < h->h_row_ptr[i + 1]; ++e) {
                const int c = h->h_col_idx[e];
                crow[fill[c]] = (int32_t)i;
                cperm[fill[c]] = (int32_t)e;
                fill[c]++;
            }
        // rows within a column are increasing because rows are visited in order
        for (int64_t c = 0; c < n; ++c)
            for (int32_t q = cptr[c] + 1; q < cptr[c + 1]; ++q)
                if (crow[q] == crow[q - 1]) {
                    delete h;
                    return create_fail("rsrr_create: duplicate entry in the pattern");
                }
        h->h_csc_ptr = std::move(cptr);
        h->h_csc_row = std::move(crow);
        h->h_csc_perm = std::move(cperm);
    }
    fill_points(h, region, N);
    rsrr_status st = fill_coef(h);
    if (st != RSRR_OK) {
        delete h;
        return st;
    }
    if (h->opts.flags & RSRR_FLAG_REAL) {
        // real arithmetic: T(z_j) = sum_i f_i(z_j) A_i real at every point
        bool ok = true;
        for (int imag : h->fn_imag) ok = ok && !imag;
        for (const cplx &zj : h->z) ok = ok && zj.imag() == 0.0;
        for (const double2 &c : h->h_coef) ok = ok && c.y == 0.0;
        if (!ok) {
            delete h;
            return create_fail("rsrr_create: RSRR_FLAG_REAL needs real values, real sampling points "
                               "and real f_i there");
        }
        if (h->opts.refine == RSRR_REFINE_GMRES) {
            delete h;
            return create_fail("rsrr_create: RSRR_FLAG_REAL does not combine with RSRR_REFINE_GMRES");
        }
        h->real = true;
    }
    *out = h;
    return RSRR_OK;
}

// device part of rsrr_create
rsrr_status Handle::allocate() { return dense ? allocate_dense() : allocate_and_upload(h_coef); }

// device bytes the handle will hold after rsrr_project and during rsrr_solve:
// its buffers (counted by a dry run of allocate()), the projection's work
// space, and rsrr_solve's temporaries (SS-FULL moment stage, eigenvector
// block of up to 256 columns)
size_t Handle::estimate_bytes() {
    dry = true;
    device_bytes = 0;
    allocate();
    dry = false;
    size_t b = device_bytes;
    device_bytes = 0;
    b += projection_ws_bytes(N * L, n, m);
    // (composite Gauss on a rectangle rounds each side to whole panels: up to
    // two more panels of 10 nodes than N_Q)
    const int nq = region.kind == RSRR_REGION_RECT ? std::max(opts.NQ + 20, 40) : opts.NQ;
    b += ssfull_dev_bytes(std::min<int64_t>((int64_t)N * L, n), m, nq, opts.KQ);
    b += sizeof(double2) * ((size_t)n + (size_t)N * L + 8) * 256 + (1u << 20);
    if (dense_terms) b += 2 * sizeof(double2) * (size_t)n * 256;  // A_i V and T(lambda) V
    return b;
}

}  // namespace rsrr

extern "C" {

rsrr_status rsrr_set_probe(rsrr_t *hh, const rsrr_c128 *U, int32_t on_device, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !U) return RSRR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double2) * (size_t)h->n * h->L;
    if (on_device) {
        CK(cudaMemcpyAsync(h->d_U, U, bytes, cudaMemcpyDeviceToDevice, s), "set_probe copy");
    } else {
        CK(cudaMemcpy(h->d_U, U, bytes, cudaMemcpyHostToDevice), "set_probe copy");
    }
    if (h->real) CK(rsrr::launch_real_part(h->d_U, (int64_t)h->n * h->L, s), "set_probe real part");
    CK(rsrr::launch_colmax(h->d_umax, h->d_U, (int)h->n, h->L, s), "set_probe colmax");
    h->sampled = false;
    h->projected = false;
    return RSRR_OK;
}

rsrr_status rsrr_sample(rsrr_t *hh, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return RSRR_EINVAL;
    rsrr_status st = h->sample((cudaStream_t)stream);
    if (st == RSRR_OK) { h->sampled = true; h->projected = false; }
    return st;
}

// Batched sampling of several band-path handles: each handle's assembly,
// then one persistent grouped band LU over every point of every handle
// (complex64 handles in one launch, complex128 ones in another; tasks
// ordered longest first), then each handle's solves and refinement.
rsrr_status rsrr_sample_batch(rsrr_t *const *handles, int32_t count, void *stream) {
    if (!handles || count < 1) {
        rsrr::thread_error() = "rsrr_sample_batch: no handles";
        return RSRR_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Handle *> hs_(count);
    for (int i = 0; i < count; ++i) {
        hs_[i] = reinterpret_cast<Handle *>(handles[i]);
        if (!hs_[i] || hs_[i]->dense || hs_[i]->real || hs_[i]->chunked()) {
            rsrr::thread_error() =
                "rsrr_sample_batch: every handle must be a complex band-path (sparse kind) handle "
                "holding the factors of all its points";
            return RSRR_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (hs_[j] == hs_[i]) {
                rsrr::thread_error() = "rsrr_sample_batch: a handle appears twice";
                return RSRR_EINVAL;
            }
    }
    for (Handle *h : hs_) {
        rsrr_status st = h->sample_band(0, h->N, s, 1);
        if (st != RSRR_OK) return st;
    }
    // the tasks: one per point, longest first (about n kl (kl + ku) each)
    std::vector<rsrr::LuTask> t64, t128;
    int kl64 = 0, kl128 = 0;
    for (Handle *h : hs_) {
        const bool mixed = h->opts.precision == RSRR_PREC_MIXED;
        const size_t ab_pt = (size_t)h->geom.ldab * h->n;
        const size_t dv_pt = (((size_t)h->n + h->geom.nb - 1) / h->geom.nb) * 2 * h->geom.nb * h->geom.nb;
        for (int pt = 0; pt < h->N; ++pt) {
            rsrr::LuTask t;
            t.ab = mixed ? (void *)(h->d_ab32 + pt * ab_pt) : (void *)(h->d_ab64 + pt * ab_pt);
            t.dinv = mixed ? (void *)(h->d_dinv32 + pt * dv_pt) : (void *)(h->d_dinv64 + pt * dv_pt);
            t.piv = h->d_piv + (size_t)pt * h->n;
            t.info = h->d_info + pt;
            t.n = (int)h->n;
            t.kl = h->kl;
            t.ku = h->ku;
            t.ldab = h->geom.ldab;
            (mixed ? t64 : t128).push_back(t);
            (mixed ? kl64 : kl128) = std::max(mixed ? kl64 : kl128, h->kl);
        }
    }
    auto work = [](const rsrr::LuTask &t) { return (double)t.n * t.kl * (double)(t.kl + t.ku + 1); };
    auto by_work = [&](const rsrr::LuTask &a, const rsrr::LuTask &b) { return work(a) > work(b); };
    std::stable_sort(t64.begin(), t64.end(), by_work);
    std::stable_sort(t128.begin(), t128.end(), by_work);
    const size_t tb = sizeof(rsrr::LuTask) * (t64.size() + t128.size());
    void *buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, tb + 256, s);
    if (e != cudaSuccess) {
        rsrr::thread_error() = std::string("rsrr_sample_batch: task table: ") + cudaGetErrorString(e);
        return RSRR_ENOMEM;
    }
    rsrr::LuTask *dt = static_cast<rsrr::LuTask *>(buf);
    int *next = reinterpret_cast<int *>(static_cast<char *>(buf) + tb);
    std::vector<rsrr::LuTask> all(t64);
    all.insert(all.end(), t128.begin(), t128.end());
    e = cudaMemcpyAsync(dt, all.data(), tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(next, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess && !t64.empty()) e = rsrr::launch_band_lu_grouped_c64(dt, (int)t64.size(), kl64, next, s);
    if (e == cudaSuccess && !t128.empty())
        e = rsrr::launch_band_lu_grouped_c128(dt + t64.size(), (int)t128.size(), kl128, next + 1, s);
    cudaError_t e2 = cudaFreeAsync(buf, s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        rsrr::thread_error() = std::string("rsrr_sample_batch: grouped band LU: ") + cudaGetErrorString(e);
        return RSRR_ECUDA;
    }
    hs_[0]->launches += (t64.empty() ? 0 : 1) + (t128.empty() ? 0 : 1);
    for (Handle *h : hs_) {
        rsrr_status st = h->sample_band(0, h->N, s, 2);
        if (st != RSRR_OK) return st;
        h->sampled = true;
        h->projected = false;
    }
    return RSRR_OK;
}

rsrr_status rsrr_add_points(rsrr_t *hh, const rsrr_c128 *z_new, int32_t count, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !z_new) return RSRR_EINVAL;
    std::vector<cplx> zz(count > 0 ? count : 0);
    for (int q = 0; q < count; ++q) zz[q] = cplx(z_new[q].re, z_new[q].im);
    rsrr_status st = h->add_points(zz.data(), count, (cudaStream_t)stream);
    if (st == RSRR_OK) h->sampled = true;
    return st;
}

rsrr_status rsrr_check(rsrr_t *hh, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return RSRR_EINVAL;
    if (!h->sampled) return h->fail(RSRR_ESTATE, "rsrr_check: no rsrr_sample yet");
    CK(cudaStreamSynchronize((cudaStream_t)stream), "rsrr_check sync");
    return h->read_outcome();
}

rsrr_status rsrr_get_samples(rsrr_t *hh, rsrr_c128 *dst, int32_t dst_on_device, void *stream) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !dst) return RSRR_EINVAL;
    if (!h->sampled) return h->fail(RSRR_ESTATE, "rsrr_get_samples: no rsrr_sample yet");
    const size_t bytes = sizeof(double2) * (size_t)h->n * h->N * h->L;
    if (dst_on_device) {
        CK(cudaMemcpyAsync(dst, h->d_X, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
           "get_samples copy");
    } else {
        CK(cudaStreamSynchronize((cudaStream_t)stream), "get_samples sync");
        CK(cudaMemcpy(dst, h->d_X, bytes, cudaMemcpyDeviceToHost), "get_samples copy");
    }
    return RSRR_OK;
}

rsrr_status rsrr_get_eta(rsrr_t *hh, double *dst) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !dst) return RSRR_EINVAL;
    if (!h->sampled) return h->fail(RSRR_ESTATE, "rsrr_get_eta: no rsrr_sample yet");
    CK(cudaDeviceSynchronize(), "get_eta sync");
    CK(cudaMemcpy(dst, h->d_eta, sizeof(double) * h->N * h->L, cudaMemcpyDeviceToHost), "get_eta");
    return RSRR_OK;
}

rsrr_status rsrr_copy_result(rsrr_t *hh, int32_t capacity, int32_t *count, rsrr_c128 *lam, double *res,
                             rsrr_c128 *V) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return RSRR_EINVAL;
    if (!h->solved) return h->fail(RSRR_ESTATE, "rsrr_copy_result: no rsrr_solve yet");
    const int32_t cnt = (int32_t)h->res_lam.size();
    if (count) *count = cnt;
    if (capacity < cnt) return h->fail(RSRR_EINVAL, "rsrr_copy_result: capacity below the eigenpair count");
    if (lam) std::copy(h->res_lam.begin(), h->res_lam.end(), lam);
    if (res) std::copy(h->res_res.begin(), h->res_res.end(), res);
    if (V) std::copy(h->res_V.begin(), h->res_V.end(), V);
    return RSRR_OK;
}

rsrr_status rsrr_get_points(rsrr_t *hh, rsrr_c128 *dst) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !dst) return RSRR_EINVAL;
    for (int j = 0; j < h->N; ++j) dst[j] = {h->z[j].real(), h->z[j].imag()};
    return RSRR_OK;
}

rsrr_status rsrr_get_stats(rsrr_t *hh, rsrr_stats *out) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h || !out) return RSRR_EINVAL;
    CK(cudaDeviceSynchronize(), "get_stats sync");
    if (h->sampled) h->read_outcome();
    if (h->timed_project) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, h->events[6], h->events[7]), "event time");
        h->stage_ms[5] = t;
        h->timed_project = false;
    }
    if (h->gemm_timed) {
        CK(h->gemm_pool.sum_pairs_ms(&h->gemm_ms), "event time");
        CK(h->tc_pool.sum_pairs_ms(&h->tc_ms), "event time");
        h->gemm_timed = false;
    }
    memset(out, 0, sizeof *out);
    out->n = h->n; out->N = h->N; out->L = h->L; out->m = h->m;
    out->kl = h->kl; out->ku = h->ku;
    out->refine_sweeps = h->stat_sweeps;
    out->converged = h->stat_converged;
    out->singular_point = h->stat_singular;
    out->max_eta = h->stat_max_eta;
    out->k = h->k;
    out->kc = h->kc;
    out->sigma1 = h->sigma1;
    out->sigmak = h->sigmak;
    out->device_bytes = h->device_bytes;
    out->launches = h->launches;
    for (int i = 0; i < 6; ++i) out->stage_ms[i] = h->stage_ms[i];
    out->gemm_flops = h->gemm_flops;
    out->gemm_ms = h->gemm_ms;
    out->tc_flops = h->tc_flops;
    out->tc_ms = h->tc_ms;
    return RSRR_OK;
}

const char *rsrr_last_error(const rsrr_t *hh) {
    const Handle *h = reinterpret_cast<const Handle *>(hh);
    if (!h) return rsrr::thread_error().c_str();
    return h->err.c_str();
}

void rsrr_destroy(rsrr_t *hh) {
    Handle *h = reinterpret_cast<Handle *>(hh);
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
namespace rsrr {

rsrr_status Handle::allocate_and_upload(const std::vector<double2> &coef) {
    Handle *h = this;
    const size_t nL = (size_t)n * L, NL = (size_t)N * L;
    CK(alloc(&d_row_ptr, n + 1), "alloc");
    CK(alloc(&d_col_idx, nnz), "alloc");
    CK(alloc(&d_vals, (size_t)m * nnz), "alloc");
    CK(alloc(&d_csc_ptr, n + 1), "alloc");
    CK(alloc(&d_csc_row, nnz), "alloc");
    CK(alloc(&d_csc_perm, nnz), "alloc");
    CK(alloc(&d_coef, (size_t)N * m), "alloc");
    CK(alloc(&d_U, nL), "alloc");
    CK(alloc(&d_umax, L), "alloc");
    CK(alloc(&d_X, nL * N), "alloc S");
    CK(alloc(&d_piv, (size_t)n * N), "alloc pivots");
    CK(alloc(&d_info, N), "alloc");
    CK(alloc(&d_tnorm, N), "alloc");
    CK(alloc(&d_eta, NL), "alloc");
    CK(alloc(&d_rmax, NL), "alloc");
    CK(alloc(&d_xmax, NL), "alloc");
    CK(alloc(&d_done, N), "alloc");
    CK(alloc(&d_sweep_flags, opts.max_refine + 2), "alloc");
    CK(alloc(&d_tmo, 1), "alloc");
    const size_t band = (size_t)geom.ldab * n * fcap;
    {
        const bool mx = opts.precision == RSRR_PREC_MIXED;
        const size_t smem2 = real ? (mx ? band_solve2_smem_r32(geom) : band_solve2_smem_r64(geom))
                                  : (mx ? band_solve2_smem_c64(geom) : band_solve2_smem_c128(geom));
        solve2 = !(opts.flags & RSRR_FLAG_PLAIN_SOLVE) && smem2 <= 227 * 1024 &&
                 geom.kl + geom.nb <= KL_MAX + 32;
        use_solve2 = solve2;
        cluster_lu = !(opts.flags & RSRR_FLAG_ONE_CTA_LU);
        if (solve2) {
            CK(alloc(&d_bperm, (size_t)fcap * ((n + geom.nb - 1) / geom.nb) * 2 * geom.nb),
               "alloc block permutations");
            CK(alloc(&d_gate, 1), "alloc");
        }
    }
    const size_t dinv_n = (size_t)fcap * ((n + geom.nb - 1) / geom.nb) * 2 * geom.nb * geom.nb;
    if (real && opts.precision == RSRR_PREC_MIXED) {
        CK(alloc(&d_abr32, band), "alloc band factors (float)");
        CK(alloc(&d_dinvr32, dinv_n), "alloc block inverses");
        CK(alloc(&d_R, nL * fcap), "alloc residual");
        CK(alloc(&d_Dr32, nL * fcap), "alloc correction");
    } else if (real) {
        CK(alloc(&d_abr64, band), "alloc band factors (double)");
        CK(alloc(&d_dinvr64, dinv_n), "alloc block inverses");
        CK(alloc(&d_Dr64, nL * fcap), "alloc real solve buffer");
    } else if (opts.precision == RSRR_PREC_MIXED) {
        CK(alloc(&d_ab32, band), "alloc band factors (complex64)");
        CK(alloc(&d_dinv32, dinv_n),
           "alloc block inverses");
        CK(alloc(&d_R, nL * fcap), "alloc residual");
        CK(alloc(&d_D, nL * fcap), "alloc correction");
    } else {
        CK(alloc(&d_ab64, band), "alloc band factors (complex128)");
        CK(alloc(&d_dinv64, dinv_n),
           "alloc block inverses");
    }
    if (dry) return RSRR_OK;
    // (pageable sources: each copy returns once its source has been staged)
    const auto H2D = cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(d_row_ptr, h_row_ptr.data(), sizeof(int32_t) * (n + 1), H2D, hs), "upload");
    CK(cudaMemcpyAsync(d_col_idx, h_col_idx.data(), sizeof(int32_t) * nnz, H2D, hs), "upload");
    CK(cudaMemcpyAsync(d_vals, h_vals.data(), sizeof(double) * m * nnz, H2D, hs), "upload");
    CK(cudaMemcpyAsync(d_csc_ptr, h_csc_ptr.data(), sizeof(int32_t) * (n + 1), H2D, hs), "upload");
    CK(cudaMemcpyAsync(d_csc_row, h_csc_row.data(), sizeof(int32_t) * nnz, H2D, hs), "upload");
    CK(cudaMemcpyAsync(d_csc_perm, h_csc_perm.data(), sizeof(int32_t) * nnz, H2D, hs), "upload");
    CK(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double2) * coef.size(), H2D, hs), "upload");
    // default probe: complex normal entries from a fixed-seed generator;
    // rsrr_set_probe replaces it
    {
        std::vector<double2> U;
        default_probe(U, nL, seed);
        CK(cudaMemcpyAsync(d_U, U.data(), sizeof(double2) * nL, H2D, hs), "upload");
    }
    if (real) CK(launch_real_part(d_U, (int64_t)nL, hs), "probe real part");
    CK(launch_colmax(d_umax, d_U, (int)n, L, hs), "colmax");
    CK(wait(), "create sync");
    dp.n = n; dp.nnz = nnz; dp.N = N; dp.L = L; dp.m = m;
    dp.row_ptr = d_row_ptr; dp.col_idx = d_col_idx; dp.vals = d_vals;
    dp.csc_ptr = d_csc_ptr; dp.csc_row = d_csc_row; dp.csc_perm = d_csc_perm;
    dp.coef = d_coef; dp.U = d_U;
    return RSRR_OK;
}

// Step 2 of RSRR on the GPU, asynchronously on stream s.
rsrr_status Handle::mark(int i, cudaStream_t s) {
    Handle *h = this;
    if (!opts.timing) return RSRR_OK;
    if (!events[0]) {
        for (auto &e : events) CK(cudaEventCreate(&e), "event");
    }
    CK(cudaEventRecord(events[i], s), "event record");
    return RSRR_OK;
}

// X = (P L U)^{-1} X in place for points p0 .. p0+np-1 not skipped (factors
// of the last LU; B and skip point at the first point of the range): the
// streaming solve when it fits, else the one-kernel solve.
cudaError_t Handle::band_solve(bool mixed, void *B, const int32_t *skip, int p0, int np, cudaStream_t s) {
    const int nn = (int)n;
    const size_t ab_pt = (size_t)geom.ldab * n;
    const size_t nblk = ((size_t)n + geom.nb - 1) / geom.nb;
    const size_t bp_pt = nblk * 2 * geom.nb, dv_pt = nblk * 2 * geom.nb * geom.nb;
    if (mixed)
        return use_solve2 ? launch_band_solve2_c64(d_ab32 + fo(p0) * ab_pt, d_bperm + fo(p0) * bp_pt, d_dinv32 + fo(p0) * dv_pt,
                                               static_cast<float2 *>(B), geom, np, nn, L, skip, s)
                      : launch_band_solve_c64(d_ab32 + fo(p0) * ab_pt, d_piv + (size_t)p0 * n, d_dinv32 + fo(p0) * dv_pt,
                                              static_cast<float2 *>(B), geom, np, nn, L, skip, s);
    return use_solve2 ? launch_band_solve2_c128(d_ab64 + fo(p0) * ab_pt, d_bperm + fo(p0) * bp_pt, d_dinv64 + fo(p0) * dv_pt,
                                            static_cast<double2 *>(B), geom, np, nn, L, skip, s)
                  : launch_band_solve_c128(d_ab64 + fo(p0) * ab_pt, d_piv + (size_t)p0 * n, d_dinv64 + fo(p0) * dv_pt,
                                           static_cast<double2 *>(B), geom, np, nn, L, skip, s);
}

// the real path's X = (P L U)^{-1} X (float B for the mixed path, double for
// the FP64 path), same choice of kernels as band_solve
cudaError_t Handle::real_solve(bool mixed, void *B, const int32_t *skip, int p0, int np, cudaStream_t s) {
    const int nn = (int)n;
    const size_t ab_pt = (size_t)geom.ldab * n;
    const size_t nblk = ((size_t)n + geom.nb - 1) / geom.nb;
    const size_t bp_pt = nblk * 2 * geom.nb, dv_pt = nblk * 2 * geom.nb * geom.nb;
    if (mixed)
        return use_solve2 ? launch_band_solve2_r32(d_abr32 + fo(p0) * ab_pt, d_bperm + fo(p0) * bp_pt, d_dinvr32 + fo(p0) * dv_pt,
                                                   static_cast<float *>(B), geom, np, nn, L, skip, s)
                          : launch_band_solve_r32(d_abr32 + fo(p0) * ab_pt, d_piv + (size_t)p0 * n, d_dinvr32 + fo(p0) * dv_pt,
                                                  static_cast<float *>(B), geom, np, nn, L, skip, s);
    return use_solve2 ? launch_band_solve2_r64(d_abr64 + fo(p0) * ab_pt, d_bperm + fo(p0) * bp_pt, d_dinvr64 + fo(p0) * dv_pt,
                                               static_cast<double *>(B), geom, np, nn, L, skip, s)
                      : launch_band_solve_r64(d_abr64 + fo(p0) * ab_pt, d_piv + (size_t)p0 * n, d_dinvr64 + fo(p0) * dv_pt,
                                              static_cast<double *>(B), geom, np, nn, L, skip, s);
}

cudaError_t Handle::sweep_solve(float2 *B, const int32_t *skip, int p0, int np, cudaStream_t s) {
    if (!use_solve2 || !d_gate || (opts.flags & RSRR_FLAG_WIDE_SOLVE_ONLY)) return band_solve(true, B, skip, p0, np, s);
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t ab_pt = (size_t)geom.ldab * n;
    const size_t nblk = ((size_t)n + geom.nb - 1) / geom.nb;
    const size_t bp_pt = nblk * 2 * geom.nb, dv_pt = nblk * 2 * geom.nb * geom.nb;
    const float2 *ab = d_ab32 + fo(p0) * ab_pt, *dv = d_dinv32 + fo(p0) * dv_pt;
    const int32_t *bp = d_bperm + fo(p0) * bp_pt;
    // the device picks the shape (16, 8, 4 or 2 right-hand sides per CTA)
    // from the points still active; the other three launches return at once
    cudaError_t e = launch_solve_gate(skip, np, L, sms, d_gate, s);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = launch_band_solve2_c64(ab, bp, dv, B, geom, np, (int)n, L, skip, s, 16 >> k, d_gate, k);
    launches += 4;
    return e;
}

// GMRES refinement (Section 4.3's X_j = T(z_j)^{-1} U to FP64 backward
// error): per cycle r = U - T X and eta (done flags), then gmres_m Arnoldi
// steps per active column: z_j = LU^{-1} v_j (complex64 solve), w = T z_j
// (FP64), modified Gram-Schmidt against v_0..v_j, v_{j+1} = w / ||w||; the
// (m+1) x m Hessenberg least-squares problem min ||beta e_1 - H y|| of every
// column is solved on the host by Givens rotations, and X += Z y.
rsrr_status Handle::refine_gmres(int p0, int np, const DevProblem &dq, cudaStream_t s) {
    Handle *h = this;
    const int m_ = opts.gmres_m, NL = N * L;
    const int64_t per_pt = (int64_t)n * L;
    const int nc = np * L;  // columns of the range
    const size_t vec = (size_t)n * NL;
    if (!d_gV) {
        CK(alloc(&d_gV, vec * (m_ + 1)), "alloc GMRES vectors");
        CK(alloc(&d_gZ, vec * m_), "alloc GMRES directions");
        CK(alloc(&d_zeroU, (size_t)per_pt), "alloc");
        CK(alloc(&d_gH, (size_t)NL * (m_ + 1) * m_), "alloc");
        CK(alloc(&d_gy, (size_t)NL * m_), "alloc");
        CK(alloc(&d_gnorm, (size_t)NL * (m_ + 1)), "alloc");
        CK(cudaMemsetAsync(d_zeroU, 0, sizeof(double2) * per_pt, s), "memset");
    }
    DevProblem d0 = dq;  // T z with a zero probe: residual kernel gives -T z
    d0.U = d_zeroU;
    int32_t *done = d_done + p0;
    double *tnorm = d_tnorm + p0, *eta = d_eta + (size_t)p0 * L;
    double *rmax = d_rmax + (size_t)p0 * L, *xmax = d_xmax + (size_t)p0 * L;
    double2 *X = d_X + p0 * per_pt, *R = d_R + fo(p0) * per_pt;
    float2 *D = d_D + fo(p0) * per_pt;
    auto Vj = [&](int j) { return d_gV + (size_t)j * vec + p0 * per_pt; };
    auto Zj = [&](int j) { return d_gZ + (size_t)j * vec + p0 * per_pt; };
    double2 *H = d_gH;        // (i, j) block of nc entries at (i m + j) NL
    double *nrm = d_gnorm;    // beta at 0, ||w_j|| at (j + 1) NL
    std::vector<int32_t> hdone(np);
    std::vector<double2> hH((size_t)NL * (m_ + 1) * m_), hy((size_t)NL * m_);
    std::vector<double> hn((size_t)NL * (m_ + 1));
    for (int it = 0; it < opts.max_refine; ++it) {
        CK(launch_residual(R, X, dq, rmax, xmax, done, s), "residual");
        CK(launch_eta(eta, done, rmax, xmax, d_umax, tnorm, np, L, opts.eta_tol, d_sweep_flags + it, done, s),
           "eta");
        CK(cudaMemcpyAsync(hdone.data(), done, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, s), "done");
        CK(cudaStreamSynchronize(s), "done sync");
        bool any = false;
        for (int q = 0; q < np; ++q) any = any || !hdone[q];
        launches += 2;
        if (!any) break;
        CK(rf_norm(R, n, nc, L, done, nrm, s), "beta");
        CK(rf_scale(Vj(0), R, nrm, n, nc, L, done, s), "v0");
        launches += 2;
        for (int j = 0; j < m_; ++j) {
            CK(launch_narrow(D, Vj(j), per_pt, np, done, s), "narrow");
            CK(sweep_solve(D, done, p0, np, s), "preconditioner");
            CK(launch_widen(Zj(j), D, per_pt * np, s), "widen");
            CK(launch_residual(R, Zj(j), d0, rmax, xmax, done, s), "T z");
            CK(rf_axpy(R, nullptr, nullptr, -1.0, n, nc, L, done, s), "w = T z");
            launches += 5;
            for (int i = 0; i <= j; ++i) {
                double2 *hij = H + (size_t)(i * m_ + j) * NL;
                CK(rf_dot(Vj(i), R, n, nc, L, done, hij, s), "h_ij");
                CK(rf_axpy(R, Vj(i), hij, 1.0, n, nc, L, done, s), "w -= h v");
                launches += 2;
            }
            CK(rf_norm(R, n, nc, L, done, nrm + (size_t)(j + 1) * NL, s), "h_j+1,j");
            CK(rf_scale(Vj(j + 1), R, nrm + (size_t)(j + 1) * NL, n, nc, L, done, s), "v_j+1");
            launches += 2;
        }
        CK(cudaMemcpyAsync(hH.data(), H, sizeof(double2) * hH.size(), cudaMemcpyDeviceToHost, s), "H");
        CK(cudaMemcpyAsync(hn.data(), nrm, sizeof(double) * hn.size(), cudaMemcpyDeviceToHost, s), "H");
        CK(cudaStreamSynchronize(s), "H sync");
        // per column: Givens QR of the (m+1) x m Hessenberg, y = R^{-1} g
        for (int c = 0; c < nc; ++c) {
            if (hdone[c / L]) continue;
            std::vector<cplx> Hc((size_t)(m_ + 1) * m_, 0.0), g(m_ + 1, 0.0);
            for (int j = 0; j < m_; ++j) {
                for (int i = 0; i <= j; ++i) {
                    const double2 v = hH[(size_t)(i * m_ + j) * NL + c];
                    Hc[(size_t)j * (m_ + 1) + i] = cplx(v.x, v.y);
                }
                Hc[(size_t)j * (m_ + 1) + j + 1] = hn[(size_t)(j + 1) * NL + c];
            }
            g[0] = hn[c];
            int kk = m_;  // columns used: up to the first (lucky) breakdown
            for (int j = 0; j < m_; ++j) {
                cplx &a = Hc[(size_t)j * (m_ + 1) + j], &b = Hc[(size_t)j * (m_ + 1) + j + 1];
                // (the rotations of steps < j were applied to this column at their step)
                const double r = std::sqrt(std::norm(a) + std::norm(b));
                if (r == 0.0) { kk = j; break; }
                const cplx cs = a / r, sn = b / r;
                // rotation G = [[conj(cs), conj(sn)], [-sn, cs]] on rows j, j+1 of columns j.. and of g
                for (int jj = j; jj < m_; ++jj) {
                    cplx &x = Hc[(size_t)jj * (m_ + 1) + j], &y2 = Hc[(size_t)jj * (m_ + 1) + j + 1];
                    const cplx t1 = std::conj(cs) * x + std::conj(sn) * y2, t2 = -sn * x + cs * y2;
                    x = t1;
                    y2 = t2;
                }
                const cplx g1 = std::conj(cs) * g[j] + std::conj(sn) * g[j + 1], g2 = -sn * g[j] + cs * g[j + 1];
                g[j] = g1;
                g[j + 1] = g2;
                if (hn[(size_t)(j + 1) * NL + c] == 0.0) { kk = j + 1; break; }
            }
            std::vector<cplx> y(m_, 0.0);
            for (int j = kk - 1; j >= 0; --j) {
                cplx acc = g[j];
                for (int jj = j + 1; jj < kk; ++jj) acc -= Hc[(size_t)jj * (m_ + 1) + j] * y[jj];
                y[j] = acc / Hc[(size_t)j * (m_ + 1) + j];
            }
            for (int j = 0; j < m_; ++j) hy[(size_t)c * m_ + j] = make_double2(y[j].real(), y[j].imag());
        }
        CK(cudaMemcpyAsync(d_gy, hy.data(), sizeof(double2) * (size_t)nc * m_, cudaMemcpyHostToDevice, s), "y");
        CK(rf_update(X, Zj(0), (int64_t)vec, d_gy, m_, n, nc, L, done, s), "X += Z y");
        CK(cudaStreamSynchronize(s), "y sync");  // the host copy of y is reused next cycle
        launches += 1;
    }
    return RSRR_OK;
}

rsrr_status Handle::sample(cudaStream_t s) {
    if (dense) return sample_dense(0, N, s);
    if ((opts.flags & RSRR_FLAG_AUTOTUNE) && !tuned && !real && !chunked()) {
        rsrr_status st = autotune(s);
        if (st != RSRR_OK) return st;
    }
    if (opts.flags & RSRR_FLAG_GRAPH) return sample_graph(s);
    return sample_range(0, N, s);
}

rsrr_status Handle::sample_range(int p0, int np, cudaStream_t s) {
    if (!chunked()) return sample_band(p0, np, s);
    // chunks of fcap points through the same band storage; the stream orders
    // each chunk's factorisation after the previous chunk's last solve
    rsrr_status st = RSRR_OK;
    for (int q = p0; q < p0 + np && st == RSRR_OK; q += fcap) {
        fbase = q;
        st = sample_band(q, std::min(fcap, p0 + np - q), s);
    }
    fbase = 0;
    return st;
}

namespace {
// the autotuner's choices per problem shape, for the whole process
struct TuneKey {
    int64_t n;
    int kl, ku, N, L, prec;
    bool operator<(const TuneKey &o) const {
        return std::tie(n, kl, ku, N, L, prec) < std::tie(o.n, o.kl, o.ku, o.N, o.L, o.prec);
    }
};
struct TuneVal {
    bool cluster, solve2;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
}  // namespace

// Times the band LU variants (cluster of two CTAs, one CTA per point; same
// factors bit for bit) and the solve variants (streaming, one-kernel) on the
// handle's own problem, keeps the faster of each, and caches the choice.
rsrr_status Handle::autotune(cudaStream_t s) {
    Handle *h = this;
    tuned = true;
    const TuneKey key{n, kl, ku, N, L, opts.precision};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            cluster_lu = it->second.cluster;
            use_solve2 = solve2 && it->second.solve2;
            return RSRR_OK;
        }
    }
    const bool mixed = opts.precision == RSRR_PREC_MIXED;
    const int nn = (int)n;
    const int64_t per_pt = (int64_t)n * L;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "tune event");
    CK(cudaEventCreate(&e1), "tune event");
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } guard{e0, e1};
    auto elapsed = [&](float *ms) {
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        return e;
    };
    float t_lu[2] = {0.f, 0.f}, t_sv[2] = {1e30f, 1e30f};
    for (int c = 0; c < 2; ++c) {  // c = 1: cluster
        if (mixed) CK(launch_assemble<float2>(d_ab32, geom, dp, s), "tune assemble");
        else CK(launch_assemble<double2>(d_ab64, geom, dp, s), "tune assemble");
        CK(cudaEventRecord(e0, s), "tune event");
        if (mixed) CK(launch_band_lu_c64(d_ab32, d_piv, d_info, d_dinv32, geom, N, nn, s, c == 1), "tune LU");
        else CK(launch_band_lu_c128(d_ab64, d_piv, d_info, d_dinv64, geom, N, nn, s, c == 1), "tune LU");
        CK(cudaEventRecord(e1, s), "tune event");
        CK(elapsed(&t_lu[c]), "tune timing");
        launches += 2;
    }
    if (solve2) {
        CK(launch_block_perm(d_bperm, d_piv, nn, geom.kl, geom.nb, N, s), "tune block permutations");
        launches += 1;
    }
    const bool save = use_solve2;
    for (int v = 0; v < (solve2 ? 2 : 1); ++v) {  // v = 1: streaming
        use_solve2 = v == 1;
        void *B = mixed ? (void *)d_D : (void *)d_X;
        if (mixed) CK(launch_broadcast_probe_c64(d_D, d_U, per_pt, N, s), "tune probe");
        else CK(launch_broadcast_probe_c128(d_X, d_U, per_pt, N, s), "tune probe");
        CK(cudaEventRecord(e0, s), "tune event");
        CK(band_solve(mixed, B, nullptr, 0, N, s), "tune solve");
        CK(cudaEventRecord(e1, s), "tune event");
        CK(elapsed(&t_sv[v]), "tune timing");
        launches += 2;
    }
    use_solve2 = save;
    const TuneVal val{t_lu[1] <= t_lu[0], solve2 && t_sv[1] <= t_sv[0]};
    cluster_lu = val.cluster;
    use_solve2 = val.solve2;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = val;
    return RSRR_OK;
}

void Handle::drop_graph() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    graph_exec = nullptr;
    graph = nullptr;
    graph_calls = 0;
}

// rsrr_sample as a CUDA graph: eager first call, capture on the second, replays after
rsrr_status Handle::sample_graph(cudaStream_t s) {
    Handle *h = this;
    if (graph_exec) {
        CK(cudaGraphLaunch(graph_exec, s), "graph launch");
        launches += graph_launches;
        timed_sample = opts.timing != 0;
        return RSRR_OK;
    }
    if (graph_failed || s == nullptr || graph_calls++ == 0) return sample_range(0, N, s);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        graph_failed = true;
        return sample_range(0, N, s);
    }
    const int64_t l0 = launches;
    const rsrr_status st = sample_range(0, N, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (st != RSRR_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        graph_failed = true;
        launches = l0;
        return sample_range(0, N, s);
    }
    graph = g;
    graph_launches = launches - l0;
    launches = l0;
    if (cudaGraphInstantiate(&graph_exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph();
        graph_failed = true;
        return sample_range(0, N, s);
    }
    CK(cudaGraphLaunch(graph_exec, s), "graph launch");
    launches += graph_launches;
    return RSRR_OK;
}

// Step 2 of RSRR on the GPU for sampling points p0 .. p0+np-1, asynchronously
// on stream s (every point for rsrr_sample; the appended points for
// rsrr_add_points, which leaves the others' samples untouched).
rsrr_status Handle::sample_band(int p0, int np, cudaStream_t s, int phase) {
    Handle *h = this;
    const int nn = (int)n;
    const int64_t per_pt = (int64_t)n * L;
    const size_t ab_pt = (size_t)geom.ldab * n;
    const size_t nblk = ((size_t)n + geom.nb - 1) / geom.nb;
    const size_t bp_pt = nblk * 2 * geom.nb, dv_pt = nblk * 2 * geom.nb * geom.nb;
    // the range's view of the problem: coefficient rows p0 .. p0+np-1
    DevProblem dq = dp;
    dq.N = np;
    dq.coef = dp.coef + (size_t)p0 * m;
    int32_t *piv = d_piv + (size_t)p0 * n, *info = d_info + p0, *done = d_done + p0;
    double *tnorm = d_tnorm + p0, *eta = d_eta + (size_t)p0 * L;
    double *rmax = d_rmax + (size_t)p0 * L, *xmax = d_xmax + (size_t)p0 * L;
    double2 *X = d_X + p0 * per_pt;
    rsrr_status ms;
    if (phase != 2) {
        CK(cudaMemsetAsync(d_tmo, 0, sizeof(unsigned int), s), "memset");
        if ((ms = mark(0, s)) != RSRR_OK) return ms;
        CK(cudaMemsetAsync(d_sweep_flags, 0, sizeof(int32_t) * (opts.max_refine + 2), s), "memset");
        if (opts.flags & RSRR_FLAG_INJECT_TIMEOUT) {
            CK(launch_wait_check(4096, d_tmo, s), "injected wait");
            launches += 1;
        }
        CK(launch_tnorm(tnorm, dq, s), "tnorm");
        if (real && opts.precision == RSRR_PREC_MIXED)
            CK(launch_assemble<float>(d_abr32 + fo(p0) * ab_pt, geom, dq, s), "assemble");
        else if (real) CK(launch_assemble<double>(d_abr64 + fo(p0) * ab_pt, geom, dq, s), "assemble");
        else if (opts.precision == RSRR_PREC_MIXED)
            CK(launch_assemble<float2>(d_ab32 + fo(p0) * ab_pt, geom, dq, s), "assemble");
        else CK(launch_assemble<double2>(d_ab64 + fo(p0) * ab_pt, geom, dq, s), "assemble");
        if ((ms = mark(1, s)) != RSRR_OK) return ms;
        if (phase == 1) return RSRR_OK;  // the caller factors (grouped LU of rsrr_sample_batch)
    }
    if (real && opts.precision == RSRR_PREC_MIXED) {
        // real float factors, FP64 complex residuals (zero imaginary parts)
        float *ab = d_abr32 + fo(p0) * ab_pt, *D = d_Dr32 + fo(p0) * per_pt;
        double2 *R = d_R + fo(p0) * per_pt;
        CK(launch_band_lu_r32(ab, piv, info, d_dinvr32 + fo(p0) * dv_pt, geom, np, nn, s, cluster_lu), "band LU");
        if (use_solve2) {
            CK(launch_block_perm(d_bperm + fo(p0) * bp_pt, piv, nn, geom.kl, geom.nb, np, s), "block permutations");
            launches += 1;
        }
        if ((ms = mark(2, s)) != RSRR_OK) return ms;
        CK(launch_broadcast_probe_r32(D, d_U, per_pt, np, s), "probe");
        CK(real_solve(true, D, nullptr, p0, np, s), "band solve");
        CK(launch_widen_r32(X, D, per_pt * np, s), "widen");
        CK(cudaMemsetAsync(done, 0, sizeof(int32_t) * np, s), "memset");
        if ((ms = mark(3, s)) != RSRR_OK) return ms;
        launches += 5;  // assemble, LU, probe, solve, widen
        for (int it = 0; it < opts.max_refine; ++it) {
            CK(launch_residual(R, X, dq, rmax, xmax, done, s), "residual");
            CK(launch_eta(eta, done, rmax, xmax, d_umax, tnorm, np, L, opts.eta_tol, d_sweep_flags + it, done, s),
               "eta");
            CK(launch_narrow_r32(D, R, per_pt, np, done, s), "narrow");
            CK(real_solve(true, D, done, p0, np, s), "band solve");
            CK(launch_update_r32(X, D, per_pt, np, done, s), "update");
            launches += 5;
        }
    } else if (real) {
        double *ab = d_abr64 + fo(p0) * ab_pt, *D = d_Dr64 + fo(p0) * per_pt;
        CK(launch_band_lu_r64(ab, piv, info, d_dinvr64 + fo(p0) * dv_pt, geom, np, nn, s, cluster_lu), "band LU");
        if (use_solve2) {
            CK(launch_block_perm(d_bperm + fo(p0) * bp_pt, piv, nn, geom.kl, geom.nb, np, s), "block permutations");
            launches += 1;
        }
        if ((ms = mark(2, s)) != RSRR_OK) return ms;
        CK(launch_broadcast_probe_r64(D, d_U, per_pt, np, s), "probe");
        CK(real_solve(false, D, nullptr, p0, np, s), "band solve");
        CK(launch_widen_r64(X, D, per_pt * np, s), "widen");
        if ((ms = mark(3, s)) != RSRR_OK) return ms;
        launches += 5;  // assemble, LU, probe, solve, widen
    } else if (opts.precision == RSRR_PREC_MIXED) {
        float2 *ab = d_ab32 + fo(p0) * ab_pt, *D = d_D + fo(p0) * per_pt;
        double2 *R = d_R + fo(p0) * per_pt;
        if (phase == 0)
            CK(launch_band_lu_c64(ab, piv, info, d_dinv32 + fo(p0) * dv_pt, geom, np, nn, s, cluster_lu), "band LU");
        if (use_solve2) {
            CK(launch_block_perm(d_bperm + fo(p0) * bp_pt, piv, nn, geom.kl, geom.nb, np, s), "block permutations");
            launches += 1;
        }
        if ((ms = mark(2, s)) != RSRR_OK) return ms;
        CK(launch_broadcast_probe_c64(D, d_U, per_pt, np, s), "probe");
        CK(band_solve(true, D, nullptr, p0, np, s), "band solve");
        CK(launch_widen(X, D, per_pt * np, s), "widen");
        CK(cudaMemsetAsync(done, 0, sizeof(int32_t) * np, s), "memset");
        if ((ms = mark(3, s)) != RSRR_OK) return ms;
        launches += 5;  // assemble, LU, probe, solve, widen
        if (opts.refine == RSRR_REFINE_GMRES) {
            if ((ms = refine_gmres(p0, np, dq, s)) != RSRR_OK) return ms;
        } else
        for (int it = 0; it < opts.max_refine; ++it) {
            CK(launch_residual(R, X, dq, rmax, xmax, done, s), "residual");
            CK(launch_eta(eta, done, rmax, xmax, d_umax, tnorm, np, L, opts.eta_tol, d_sweep_flags + it, done, s),
               "eta");
            CK(launch_narrow(D, R, per_pt, np, done, s), "narrow");
            CK(sweep_solve(D, done, p0, np, s), "band solve");
            CK(launch_update(X, D, per_pt, np, done, s), "update");
            launches += 5;
        }
    } else {
        double2 *ab = d_ab64 + fo(p0) * ab_pt;
        if (phase == 0)
            CK(launch_band_lu_c128(ab, piv, info, d_dinv64 + fo(p0) * dv_pt, geom, np, nn, s, cluster_lu), "band LU");
        if (use_solve2) {
            CK(launch_block_perm(d_bperm + fo(p0) * bp_pt, piv, nn, geom.kl, geom.nb, np, s), "block permutations");
            launches += 1;
        }
        if ((ms = mark(2, s)) != RSRR_OK) return ms;
        CK(launch_broadcast_probe_c128(X, d_U, per_pt, np, s), "probe");
        CK(band_solve(false, X, nullptr, p0, np, s), "band solve");
        if ((ms = mark(3, s)) != RSRR_OK) return ms;
        launches += 4;  // assemble, LU, probe, solve
    }
    if ((ms = mark(4, s)) != RSRR_OK) return ms;
    // final backward errors of every column of the range (statistics and
    // convergence).  After iterative refinement a point flagged done was not
    // corrected after the residual that flagged it, so its backward errors
    // are final: only the points corrected in the last sweep are recomputed
    const bool ir = opts.precision == RSRR_PREC_MIXED && opts.refine == RSRR_REFINE_IR && opts.max_refine > 0;
    const int32_t *fskip = ir ? done : nullptr;
    CK(launch_residual(nullptr, X, dq, rmax, xmax, fskip, s), "residual");
    CK(launch_eta(eta, done, rmax, xmax, d_umax, tnorm, np, L, opts.eta_tol,
                  d_sweep_flags + opts.max_refine + 1, fskip, s), "eta");
    if ((ms = mark(5, s)) != RSRR_OK) return ms;
    launches += 3;  // tnorm, final residual, final eta
    timed_sample = opts.timing != 0;
    return RSRR_OK;
}

// frees one buffer obtained by alloc() and forgets it
void Handle::release(void *p, size_t bytes) {
    if (!p) return;
    for (size_t q = 0; q < allocations.size(); ++q)
        if (allocations[q] == p) {
            allocations.erase(allocations.begin() + q);
            break;
        }
    raw_free(p);
    device_bytes -= std::min(device_bytes, bytes);
}

// a per-point buffer grown from N0 to N1 points of `per` elements; with keep,
// the first N0 points' contents are copied (bit for bit)
template <typename T>
cudaError_t Handle::regrow(T **p, size_t per, int N0, int N1, bool keep) {
    T *q = nullptr;
    cudaError_t e = alloc(&q, per * N1);
    if (e != cudaSuccess) return e;
    if (keep && *p && per * N0 > 0) {
        e = cudaMemcpyAsync(q, *p, sizeof(T) * per * N0, cudaMemcpyDeviceToDevice, hs);
        if (e == cudaSuccess) e = wait();
        if (e != cudaSuccess) return e;
    }
    release(*p, sizeof(T) * per * N0);
    *p = q;
    return cudaSuccess;
}

// Two-stage sampling (Section 5.4): the points z_new are appended to the
// handle's sampling points and only they are assembled, factored, solved and
// refined; the samples X_j of the earlier points stay resident, unchanged.
rsrr_status Handle::add_points(const cplx *znew, int count, cudaStream_t s) {
    Handle *h = this;
    if (!sampled) return fail(RSRR_ESTATE, "rsrr_add_points: no rsrr_sample yet");
    if (real) return fail(RSRR_EINVAL, "rsrr_add_points: not on a RSRR_FLAG_REAL handle");
    if (count < 1) return fail(RSRR_EINVAL, "rsrr_add_points: count must be >= 1");
    for (int q = 0; q < count; ++q)
        if (!std::isfinite(znew[q].real()) || !std::isfinite(znew[q].imag()))
            return fail(RSRR_EINVAL, "rsrr_add_points: points must be finite");
    if ((int64_t)N + count > (int64_t)INT32_MAX / std::max(1, L))
        return fail(RSRR_EINVAL, "rsrr_add_points: too many points");
    std::vector<cplx> fnew;
    if (!dense || dense_terms) {
        rsrr_status st = eval_terms(znew, count, fnew);
        if (st != RSRR_OK) return st;
    }
    CK(cudaStreamSynchronize(s), "add_points sync");
    CK(wait(), "add_points sync");
    const int N0 = N, N1 = N + count;
    const size_t per_pt = (size_t)n * L;
    const bool mixed = opts.precision == RSRR_PREC_MIXED;
    // kept: the samples, their backward errors, the pivot status, the
    // coefficient rows / points; the rest is work space of the next sampling
    CK(regrow(&d_X, per_pt, N0, N1, true), "regrow S");
    CK(regrow(&d_eta, (size_t)L, N0, N1, true), "regrow");
    CK(regrow(&d_info, 1, N0, N1, true), "regrow");
    CK(regrow(&d_piv, (size_t)n, N0, N1, false), "regrow");
    CK(regrow(&d_tnorm, 1, N0, N1, false), "regrow");
    CK(regrow(&d_rmax, (size_t)L, N0, N1, false), "regrow");
    CK(regrow(&d_xmax, (size_t)L, N0, N1, false), "regrow");
    CK(regrow(&d_done, 1, N0, N1, false), "regrow");
    const bool grow_factors = !chunked();  // chunked: the new points reuse the chunk storage
    if (d_R && grow_factors) CK(regrow(&d_R, per_pt, N0, N1, false), "regrow");
    if (d_D && grow_factors) CK(regrow(&d_D, per_pt, N0, N1, false), "regrow");
    if (!dense || dense_terms) CK(regrow(&d_coef, (size_t)m, N0, N1, true), "regrow");
    if (dense) {
        const size_t nn2 = (size_t)n * n;
        const int nb = mixed ? NB_C64 : NB_C128;
        const size_t dv_pt = (((size_t)n + nb - 1) / nb) * 2 * nb * nb;
        CK(regrow(&d_z, 1, N0, N1, true), "regrow");
        CK(regrow(&d_T64, nn2, N0, N1, false), "regrow dense matrices");
        if (mixed) {
            CK(regrow(&d_A32, nn2, N0, N1, false), "regrow dense factors");
            CK(regrow(&d_dinv32, dv_pt, N0, N1, false), "regrow");
        } else {
            CK(regrow(&d_ab64, nn2, N0, N1, false), "regrow dense factors");
            CK(regrow(&d_dinv64, dv_pt, N0, N1, false), "regrow");
        }
    } else if (grow_factors) {
        const size_t ab_pt = (size_t)geom.ldab * n;
        const size_t nblk = ((size_t)n + geom.nb - 1) / geom.nb;
        if (mixed) {
            CK(regrow(&d_ab32, ab_pt, N0, N1, false), "regrow band factors");
            CK(regrow(&d_dinv32, nblk * 2 * geom.nb * geom.nb, N0, N1, false), "regrow");
        } else {
            CK(regrow(&d_ab64, ab_pt, N0, N1, false), "regrow band factors");
            CK(regrow(&d_dinv64, nblk * 2 * geom.nb * geom.nb, N0, N1, false), "regrow");
        }
        if (d_bperm) CK(regrow(&d_bperm, nblk * 2 * geom.nb, N0, N1, false), "regrow");
    }
    if (grow_factors) fcap = N1;
    drop_graph();  // the captured launches name the old buffers
    // the projection's work space is sized by N L: rebuilt by the next rsrr_project
    if (proj_ws) {
        release(proj_ws, proj_ws_bytes);
        proj_ws = nullptr;
        proj_ws_bytes = 0;
        d_Q = nullptr;
        d_P = nullptr;
    }
    // the new points and their coefficient rows
    std::vector<double2> zs(count);
    for (int q = 0; q < count; ++q) zs[q] = make_double2(znew[q].real(), znew[q].imag());
    if (dense && !dense_terms)
        CK(cudaMemcpyAsync(d_z + N0, zs.data(), sizeof(double2) * count, cudaMemcpyHostToDevice, hs), "upload");
    if (!fnew.empty()) {
        std::vector<double2> cf(fnew.size());
        for (size_t e = 0; e < cf.size(); ++e) cf[e] = make_double2(fnew[e].real(), fnew[e].imag());
        CK(cudaMemcpyAsync(d_coef + (size_t)N0 * m, cf.data(), sizeof(double2) * cf.size(), cudaMemcpyHostToDevice,
                           hs), "upload");
    }
    CK(wait(), "upload sync");
    z.insert(z.end(), znew, znew + count);
    points_added = true;
    N = N1;
    dp.N = N1;
    dp.coef = d_coef;
    projected = false;
    solved = false;
    return dense ? sample_dense(N0, count, s) : sample_range(N0, count, s);
}

rsrr_status Handle::read_outcome() {
    Handle *h = this;
    // unknown until read back: a failed copy below leaves NaN, not a stale value
    stat_max_eta = std::numeric_limits<double>::quiet_NaN();
    stat_converged = 0;
    std::vector<int32_t> info(N), flags(opts.max_refine + 2);
    std::vector<double> eta((size_t)N * L);
    const auto D2H = cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(info.data(), d_info, sizeof(int32_t) * N, D2H, hs), "outcome");
    CK(cudaMemcpyAsync(flags.data(), d_sweep_flags, sizeof(int32_t) * flags.size(), D2H, hs), "outcome");
    CK(cudaMemcpyAsync(eta.data(), d_eta, sizeof(double) * eta.size(), D2H, hs), "outcome");
    CK(cudaStreamSynchronize(hs), "outcome");
    stat_singular = -1;
    for (int j = 0; j < N; ++j)
        if (info[j] != 0) { stat_singular = j; break; }
    stat_sweeps = 0;
    if (opts.precision == RSRR_PREC_MIXED)
        for (int it = 0; it < opts.max_refine; ++it) stat_sweeps += flags[it] ? 1 : 0;
    stat_max_eta = 0.0;
    bool finite = true;
    for (double e : eta) {
        if (!std::isfinite(e)) finite = false;
        stat_max_eta = std::max(stat_max_eta, e);
    }
    stat_converged = (finite && stat_max_eta <= opts.eta_tol) ? 1 : 0;
    if (!finite) stat_max_eta = std::numeric_limits<double>::quiet_NaN();
    // the stage times after the outcome, so that a failed timing query never
    // leaves the statistics of an earlier sampling in place (-1: not timed)
    if (timed_sample) {
        const int pairs[5][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}};
        for (int i = 0; i < 5; ++i) {
            float t = -1.f;
            if (cudaEventElapsedTime(&t, events[pairs[i][0]], events[pairs[i][1]]) != cudaSuccess) {
                cudaGetLastError();
                t = -1.f;
            }
            stage_ms[i] = t;
        }
        timed_sample = false;
    }
    if (stat_singular >= 0) {
        char buf[128];
        snprintf(buf, sizeof buf, "zero pivot at sampling point %d (column %d)", stat_singular,
                 info[stat_singular] - 1);
        return fail(RSRR_ESINGULAR, buf);
    }
    if (!stat_converged && opts.precision == RSRR_PREC_MIXED) {
        char buf[128];
        snprintf(buf, sizeof buf, "refinement stopped at max eta %.3e > %.1e", stat_max_eta, opts.eta_tol);
        return fail(RSRR_ENOCONV, buf);
    }
    return RSRR_OK;
}

}  // namespace rsrr

// ---------------------------------------------------------------------------
// dense (Helmholtz kernel) problems
// ---------------------------------------------------------------------------
namespace rsrr {

rsrr_status prepare_dense(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                          const rsrr_opts *opts, Handle **out) {
    if (!nep->points) return create_fail("rsrr_create: Helmholtz kind without points");
    if (!(std::isfinite(nep->diag))) return create_fail("rsrr_create: diag is not finite");
    const int64_t n = nep->n;
    if (n > 65536) return create_fail("rsrr_create: dense order above 65536");
    Handle *h = new_handle(nep, region, N, L, opts);
    if (!h) { thread_error() = "rsrr_create: out of host memory"; return RSRR_ENOMEM; }
    h->dense = true;
    h->nnz = 0;
    h->diag = nep->diag;
    h->h_points.assign(nep->points, nep->points + 3 * n);
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(h->h_points[3 * i]) || !std::isfinite(h->h_points[3 * i + 1]) ||
            !std::isfinite(h->h_points[3 * i + 2])) {
            delete h;
            return create_fail("rsrr_create: point coordinates must be finite");
        }
        for (int64_t j = 0; j < i; ++j) {
            const double dx = h->h_points[3 * i] - h->h_points[3 * j];
            const double dy = h->h_points[3 * i + 1] - h->h_points[3 * j + 1];
            const double dz = h->h_points[3 * i + 2] - h->h_points[3 * j + 2];
            const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r > 0.0)) {
                delete h;
                return create_fail("rsrr_create: two points coincide");
            }
            rmax = std::max(rmax, r);
        }
    }
    // Taylor terms about the centre: smallest P with (r_max rho)^P / P! < 1e-17;
    // the held terms are the powers (z - c)^p
    // (the region's radius about the centre: the half-diagonal of a rectangle)
    const double x = rmax * (region->kind == RSRR_REGION_RECT ? std::hypot(region->a, region->b)
                                                              : std::max(region->a, region->b));
    int P = 0;
    double term = 1.0;
    while (term >= 1e-17 && P < 200) { ++P; term *= x / P; }
    h->m = P;
    for (int p = 0; p < P; ++p) {
        rsrr_fn f{};
        f.kind = RSRR_F_TAYLOR;
        f.power = p;
        f.scale = rsrr_c128{1.0, 0.0};
        f.shift = region->center;
        h->fn.push_back(f);
        h->fn_src.push_back(p);
        h->fn_imag.push_back(0);
    }
    fill_points(h, region, N);
    *out = h;
    return RSRR_OK;
}

// T(z) = sum_i f_i(z) A_i with dense caller-supplied A_i
rsrr_status prepare_dense_terms(const rsrr_nep *nep, const rsrr_region *region, int32_t N, int32_t L,
                                const rsrr_opts *opts, Handle **out) {
    const int64_t n = nep->n;
    if (n > 32768) return create_fail("rsrr_create: dense order above 32768");
    if (!nep->dense) return create_fail("rsrr_create: dense kind without matrices");
    for (int i = 0; i < nep->m; ++i)
        if (!nep->dense[i]) return create_fail("rsrr_create: dense kind with a NULL matrix");
    Handle *h = new_handle(nep, region, N, L, opts);
    if (!h) { thread_error() = "rsrr_create: out of host memory"; return RSRR_ENOMEM; }
    h->dense = true;
    h->dense_terms = true;
    h->nnz = 0;
    h->m = nep->m;
    const size_t nn2 = (size_t)n * n;
    try {
        h->h_Aterms.resize(nn2 * nep->m);
    } catch (...) {
        delete h;
        thread_error() = "rsrr_create: out of host memory";
        return RSRR_ENOMEM;
    }
    h->a1.assign(nep->m, 0.0);
    for (int i = 0; i < nep->m; ++i) {
        const rsrr_c128 *A = nep->dense[i];
        double2 *dst = h->h_Aterms.data() + nn2 * i;
        for (int64_t c = 0; c < n; ++c) {
            double cs = 0.0;
            for (int64_t r = 0; r < n; ++r) {
                const rsrr_c128 v = A[c * n + r];
                if (!std::isfinite(v.re) || !std::isfinite(v.im)) {
                    delete h;
                    return create_fail("rsrr_create: dense matrix entries must be finite");
                }
                dst[c * n + r] = make_double2(v.re, v.im);
                cs += std::hypot(v.re, v.im);
            }
            h->a1[i] = std::max(h->a1[i], cs);
        }
        h->fn.push_back(nep->fn[i]);
        h->fn_src.push_back(i);
        h->fn_imag.push_back(0);
    }
    fill_points(h, region, N);
    rsrr_status st = fill_coef(h);
    if (st != RSRR_OK) {
        delete h;
        return st;
    }
    *out = h;
    return RSRR_OK;
}

rsrr_status Handle::allocate_dense() {
    Handle *h = this;
    const size_t nL = (size_t)n * L, NL = (size_t)N * L, nn2 = (size_t)n * n;
    const bool mixed = opts.precision == RSRR_PREC_MIXED;
    const int nb = mixed ? NB_C64 : NB_C128;
    const size_t nblk = ((size_t)n + nb - 1) / nb;
    if (dense_terms) {
        CK(alloc(&d_Aterms, (size_t)m * nn2), "alloc dense terms");
        CK(alloc(&d_coef, (size_t)N * m), "alloc");
    } else {
        CK(alloc(&d_points, 3 * n), "alloc");
    }
    CK(alloc(&d_z, N), "alloc");
    CK(alloc(&d_U, nL), "alloc");
    CK(alloc(&d_umax, L), "alloc");
    CK(alloc(&d_X, nL * N), "alloc S");
    CK(alloc(&d_R, nL * fcap), "alloc residual");
    CK(alloc(&d_piv, (size_t)n * N), "alloc pivots");
    CK(alloc(&d_info, N), "alloc");
    CK(alloc(&d_tnorm, N), "alloc");
    CK(alloc(&d_eta, NL), "alloc");
    CK(alloc(&d_rmax, NL), "alloc");
    CK(alloc(&d_xmax, NL), "alloc");
    CK(alloc(&d_done, N), "alloc");
    CK(alloc(&d_sweep_flags, opts.max_refine + 2), "alloc");
    CK(alloc(&d_tmo, 1), "alloc");
    CK(alloc(&d_T64, nn2 * N), "alloc dense matrices (complex128)");
    // the FP64 residuals U - T X (n x n times n x L per point) are FP64-accurate
    // tensor-core products when the GEMM method allows them
    if (dense_residual_sliced()) {
        dws_bytes = ozaki_workspace_bytes((int)n, L, (int)n, false);
        CK(raw_alloc(&d_dws, dws_bytes), "alloc residual product work space");
    }
    if (mixed) {
        CK(alloc(&d_A32, nn2 * N), "alloc dense factors (complex64)");
        CK(alloc(&d_D, nL * fcap), "alloc correction");
        CK(alloc(&d_dinv32, (size_t)N * nblk * 2 * nb * nb), "alloc block inverses");
    } else {
        CK(alloc(&d_ab64, nn2 * N), "alloc dense factors (complex128)");
        CK(alloc(&d_dinv64, (size_t)N * nblk * 2 * nb * nb), "alloc block inverses");
    }
    if (dry) return RSRR_OK;
    std::vector<double2> zs(N);
    for (int j = 0; j < N; ++j) zs[j] = make_double2(z[j].real(), z[j].imag());
    if (dense_terms) {
        CK(cudaMemcpyAsync(d_Aterms, h_Aterms.data(), sizeof(double2) * h_Aterms.size(), cudaMemcpyHostToDevice, hs),
           "upload");
        CK(cudaMemcpyAsync(d_coef, h_coef.data(), sizeof(double2) * h_coef.size(), cudaMemcpyHostToDevice, hs),
           "upload");
    } else {
        CK(cudaMemcpyAsync(d_points, h_points.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, hs),
           "upload");
    }
    CK(cudaMemcpyAsync(d_z, zs.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, hs), "upload");
    {
        std::vector<double2> U;
        default_probe(U, nL, seed);
        CK(cudaMemcpyAsync(d_U, U.data(), sizeof(double2) * nL, cudaMemcpyHostToDevice, hs), "upload");
    }
    CK(launch_colmax(d_umax, d_U, (int)n, L, hs), "colmax");
    CK(wait(), "create sync");
    if (dense_terms) std::vector<double2>().swap(h_Aterms);  // the device copy is the one used
    dp.n = n; dp.N = N; dp.L = L; dp.m = m; dp.U = d_U; dp.coef = d_coef;
    return RSRR_OK;
}

// whether the residual products of the dense path use the sliced tensor-core
// GEMM: by the GEMM method, AUTO for products of at least 2^30 flops
bool Handle::dense_residual_sliced() const {
    const double flops = 8.0 * (double)n * (double)L * (double)n;
    return opts.gemm == RSRR_GEMM_OZAKI || opts.gemm == RSRR_GEMM_OZAKI_MMA ||
           (opts.gemm == RSRR_GEMM_AUTO && flops >= 1073741824.0);
}

// R = U - T X in FP64 (stored complex128 T) and the column maxima of |R|, |X|,
// for points p0 .. p0+np-1, or (skip_done) only for those whose done flag is 0
// (the flags are read on the host first).
rsrr_status Handle::dense_residual(bool skip_done, int p0, int np, cudaStream_t s) {
    Handle *h = this;
    std::vector<int32_t> done(np, 0);
    if (skip_done) {
        CK(cudaMemcpyAsync(done.data(), d_done + p0, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, s), "done");
        CK(cudaStreamSynchronize(s), "done sync");
    }
    const size_t per = (size_t)n * L, nn2 = (size_t)n * n;
    for (int q = 0; q < np; ++q) {
        if (done[q]) continue;
        const size_t pt = (size_t)p0 + q;
        CK(cudaMemcpyAsync(d_R + pt * per, d_U, sizeof(double2) * per, cudaMemcpyDeviceToDevice, s), "R = U");
        if (dense_residual_sliced())
            CK(ozaki_zgemm((int)n, L, (int)n, false, d_T64 + pt * nn2, n, d_X + pt * per, n, d_R + pt * per, n,
                           -1.0, 1.0, false, d_dws, dws_bytes, s, &launches, nullptr, nullptr,
                           opts.gemm == RSRR_GEMM_OZAKI_MMA, d_tmo), "R -= T X");
        else
            CK(fp64_gemm((int)n, L, (int)n, false, d_T64 + pt * nn2, n, d_X + pt * per, n, d_R + pt * per, n,
                         -1.0, 1.0, s), "R -= T X");
        CK(launch_dense_colmax(d_R + pt * per, d_X + pt * per, (int)n, L, d_rmax + pt * L, d_xmax + pt * L, s),
           "colmax");
        launches += 2;
    }
    return RSRR_OK;
}

// Step 2 of RSRR for the dense problems, points p0 .. p0+np-1.
rsrr_status Handle::sample_dense(int p0, int np, cudaStream_t s) {
    Handle *h = this;
    const int nn = (int)n;
    const bool mixed = opts.precision == RSRR_PREC_MIXED;
    const int nb = mixed ? NB_C64 : NB_C128;
    const size_t nn2 = (size_t)n * n;
    const size_t dv_pt = (((size_t)n + nb - 1) / nb) * 2 * nb * nb;
    const int64_t per_pt = (int64_t)n * L, total = (int64_t)nn2 * np;
    int32_t *piv = d_piv + (size_t)p0 * n, *info = d_info + p0, *done = d_done + p0;
    double *tnorm = d_tnorm + p0, *eta = d_eta + (size_t)p0 * L;
    double *rmax = d_rmax + (size_t)p0 * L, *xmax = d_xmax + (size_t)p0 * L;
    double2 *X = d_X + p0 * per_pt, *T64 = d_T64 + p0 * nn2;
    rsrr_status ms;
    CK(cudaMemsetAsync(d_tmo, 0, sizeof(unsigned int), s), "memset");
    if ((ms = mark(0, s)) != RSRR_OK) return ms;
    CK(cudaMemsetAsync(d_sweep_flags, 0, sizeof(int32_t) * (opts.max_refine + 2), s), "memset");
    if (opts.flags & RSRR_FLAG_INJECT_TIMEOUT) {
        CK(launch_wait_check(4096, d_tmo, s), "injected wait");
        launches += 1;
    }
    if (dense_terms)
        CK(launch_assemble_dense_terms(T64, d_Aterms, d_coef + (size_t)p0 * m, nn, np, m, s), "assemble");
    else
        CK(launch_assemble_dense_c128(T64, d_points, d_z + p0, diag, nn, np, s), "assemble");
    CK(launch_dense_tnorm(tnorm, T64, nn, np, s), "tnorm");
    launches += 2;
    if (mixed) {
        float2 *A32 = d_A32 + p0 * nn2, *D = d_D + fo(p0) * per_pt;
        CK(launch_narrow_all(A32, T64, total, s), "narrow");
        launches += 1;
        if ((ms = mark(1, s)) != RSRR_OK) return ms;
        CK(launch_dense_lu_c64(A32, piv, info, d_dinv32 + fo(p0) * dv_pt, nn, np, s, &launches, d_tmo,
                               !(opts.flags & RSRR_FLAG_SIMT_DENSE_UPDATE)), "dense LU");
        if ((ms = mark(2, s)) != RSRR_OK) return ms;
        CK(launch_broadcast_probe_c64(D, d_U, per_pt, np, s), "probe");
        CK(launch_dense_solve_c64(A32, piv, d_dinv32 + fo(p0) * dv_pt, D, nn, np, L, nullptr, s), "dense solve");
        CK(launch_widen(X, D, per_pt * np, s), "widen");
        CK(cudaMemsetAsync(done, 0, sizeof(int32_t) * np, s), "memset");
        launches += 3;
        if ((ms = mark(3, s)) != RSRR_OK) return ms;
        for (int it = 0; it < opts.max_refine; ++it) {
            if ((ms = dense_residual(true, p0, np, s)) != RSRR_OK) return ms;
            CK(launch_eta(eta, done, rmax, xmax, d_umax, tnorm, np, L, opts.eta_tol, d_sweep_flags + it, done, s),
               "eta");
            CK(launch_narrow(D, d_R + fo(p0) * per_pt, per_pt, np, done, s), "narrow");
            CK(launch_dense_solve_c64(A32, piv, d_dinv32 + fo(p0) * dv_pt, D, nn, np, L, done, s), "dense solve");
            CK(launch_update(X, D, per_pt, np, done, s), "update");
            launches += 4;
        }
    } else {
        double2 *A64 = d_ab64 + p0 * nn2;
        CK(cudaMemcpyAsync(A64, T64, sizeof(double2) * total, cudaMemcpyDeviceToDevice, s), "copy");
        if ((ms = mark(1, s)) != RSRR_OK) return ms;
        CK(launch_dense_lu_c128(A64, piv, info, d_dinv64 + fo(p0) * dv_pt, nn, np, s, &launches), "dense LU");
        if ((ms = mark(2, s)) != RSRR_OK) return ms;
        CK(launch_broadcast_probe_c128(X, d_U, per_pt, np, s), "probe");
        CK(launch_dense_solve_c128(A64, piv, d_dinv64 + fo(p0) * dv_pt, X, nn, np, L, nullptr, s), "dense solve");
        launches += 2;
        if ((ms = mark(3, s)) != RSRR_OK) return ms;
    }
    if ((ms = mark(4, s)) != RSRR_OK) return ms;
    if ((ms = dense_residual(false, p0, np, s)) != RSRR_OK) return ms;
    CK(launch_eta(eta, done, rmax, xmax, d_umax, tnorm, np, L, opts.eta_tol, d_sweep_flags + opts.max_refine + 1,
                  nullptr, s), "eta");
    launches += 1;
    if ((ms = mark(5, s)) != RSRR_OK) return ms;
    timed_sample = opts.timing != 0;
    return RSRR_OK;
}

}  // namespace rsrr
