// Request server: continuous batching of whole RSRR solves (steps 1-5 of
// Section 4.3) on one GPU.
//
// A request is prepared on the submitting thread (descriptors validated and
// copied, sampling points and f_i(z_j) computed, device bytes estimated) and
// queued.  `slots` worker threads, each with its own non-blocking CUDA stream,
// admit queued requests in arrival order as soon as a slot is free and the
// request's bytes fit in what the memory budget has left; a later request
// may pass one that does not fit yet, at most kMaxBypass times, after which
// the waiting request is admitted next.  An admitted request allocates from
// a stream-ordered memory pool on its worker's stream, runs sample, project
// and solve, and copies its eigenpairs to host memory.  The kernels of one
// request overlap on the device with the kernels and the host work of the
// others.  Without `keep`, the request's device memory goes back to the pool
// (and its bytes to the budget) when it finishes; with `keep`, its handle
// (factors, S, Q, P_i) stays resident until release.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "admission.h"
#include "rsrr.h"
#include "rsrr_handle.h"

namespace rsrr {

constexpr int kMaxBypass = 8;

struct Request {
    int64_t id = 0, n = 0;
    Handle *h = nullptr;
    std::vector<double2> U;  // caller's probe, or empty for the default one
    size_t bytes = 0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int bypassed = 0;
    bool done = false;
    rsrr_status status = RSRR_OK;
    std::string error;
    int32_t count = 0, nbar = 0, k = 0, sweeps = 0;
    double gmax = 0.0, max_eta = 0.0;
    double t_sample = 0.0, t_project = 0.0, t_solve = 0.0;  // wall seconds of the stages
    std::vector<rsrr_c128> lam, V;
    std::vector<double> res;
    bool holds_budget = false;
};

struct Server {
    rsrr_server_opts o = {};
    int device = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, Request *> reqs;
    int64_t next_id = 1;
    size_t used = 0, peak_used = 0;
    int active = 0, peak_active = 0;
    int64_t submitted = 0, completed = 0, failed = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // the request admit_index picks; the requests it passed over count one
    // more bypass; reserves its bytes and removes it from the queue (mu held)
    Request *pick_locked() {
        const int q = admit_index(
            (int)queue.size(), [this](int i) { return queue[i]->bytes; },
            [this](int i) { return queue[i]->bypassed; }, used, (size_t)o.mem_budget_bytes, active, o.slots,
            kMaxBypass);
        if (q < 0) return nullptr;
        Request *r = queue[q];
        for (int e = 0; e < q; ++e) queue[e]->bypassed++;
        queue.erase(queue.begin() + q);
        used += r->bytes;
        peak_used = std::max(peak_used, used);
        active++;
        peak_active = std::max(peak_active, active);
        r->holds_budget = true;
        r->t_admit = now();
        return r;
    }

    void run(Request *r, cudaStream_t s) {
        Handle *h = r->h;
        h->hs = s;
        h->pool = pool;
        rsrr_status st = h->allocate();
        if (st == RSRR_OK && !r->U.empty()) {
            const size_t bytes = sizeof(double2) * r->U.size();
            cudaError_t e = cudaMemcpyAsync(h->d_U, r->U.data(), bytes, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = launch_colmax(h->d_umax, h->d_U, (int)h->n, h->L, s);
            if (e != cudaSuccess) st = h->fail(RSRR_ECUDA, "probe upload", e);
        }
        const double ta = now();
        if (st == RSRR_OK) st = h->sample(s);
        if (st == RSRR_OK) {
            h->sampled = true;
            cudaError_t e = cudaStreamSynchronize(s);
            st = e == cudaSuccess ? h->read_outcome() : h->fail(RSRR_ECUDA, "sample", e);
        }
        const double tb = now();
        if (st == RSRR_OK) {
            st = h->project(s);
            h->projected = st == RSRR_OK;
            if (st == RSRR_OK) {
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) st = h->fail(RSRR_ECUDA, "project", e);
            }
        }
        const double tc = now();
        r->t_sample = tb - ta;
        r->t_project = tc - tb;
        if (st == RSRR_OK) {
            rsrr_result res = {};
            st = h->solve(&res);
            r->t_solve = now() - tc;
            if (st >= 0) {
                r->count = res.count;
                r->nbar = res.nbar;
                r->gmax = res.gmax;
                r->lam.assign(res.lam, res.lam + res.count);
                r->res.assign(res.res, res.res + res.count);
                r->V.assign(res.V, res.V + (size_t)h->n * res.count);
            }
        }
        r->k = h->k;
        r->sweeps = h->stat_sweeps;
        r->max_eta = h->stat_max_eta;
        r->status = st;
        if (st < 0) r->error = h->err;
        cudaStreamSynchronize(s);
        if (!o.keep || st < 0) {
            delete h;  // frees into the pool, ordered on s
            cudaStreamSynchronize(s);
            r->h = nullptr;
        } else {
            h->hs = nullptr;  // later calls on the kept handle use the caller's streams
        }
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t s = nullptr;
        const bool have_stream = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            Request *r = nullptr;
            cv_work.wait(lk, [&] { return stopping || (r = pick_locked()) != nullptr; });
            if (!r) break;
            lk.unlock();
            if (have_stream) {
                run(r, s);
            } else {
                r->status = RSRR_ECUDA;
                r->error = "rsrr_server: no CUDA stream";
            }
            lk.lock();
            r->t_done = now();
            r->done = true;
            active--;
            if (!r->h) {
                used -= r->bytes;
                r->holds_budget = false;
            }
            if (r->status < 0) failed++;
            else completed++;
            cv_done.notify_all();
            cv_work.notify_all();
        }
        lk.unlock();
        if (have_stream) cudaStreamDestroy(s);
    }
};

}  // namespace rsrr

using rsrr::Handle;
using rsrr::Request;
using rsrr::Server;

static rsrr_status server_fail(rsrr_status st, const std::string &msg) {
    rsrr::thread_error() = msg;
    return st;
}

extern "C" {

void rsrr_server_opts_default(rsrr_server_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->slots = 4;
    o->keep = 0;
    o->mem_budget_bytes = (int64_t)150 * 1000 * 1000 * 1000;
    o->device = -1;
}

rsrr_status rsrr_server_create(const rsrr_server_opts *opts, rsrr_server_t **out) {
    if (!out) return server_fail(RSRR_EINVAL, "rsrr_server_create: out is NULL");
    *out = nullptr;
    Server *sv = new (std::nothrow) Server();
    if (!sv) return server_fail(RSRR_ENOMEM, "rsrr_server_create: out of host memory");
    if (opts) sv->o = *opts;
    else rsrr_server_opts_default(&sv->o);
    if (sv->o.slots < 1 || sv->o.slots > 64 || sv->o.mem_budget_bytes <= 0) {
        delete sv;
        return server_fail(RSRR_EINVAL, "rsrr_server_create: slots must be 1..64 and the budget > 0");
    }
    cudaError_t e = cudaSuccess;
    if (sv->o.device < 0) e = cudaGetDevice(&sv->device);
    else sv->device = sv->o.device;
    if (e == cudaSuccess) e = cudaSetDevice(sv->device);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = sv->device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&sv->pool, &props);
    if (e == cudaSuccess) {
        // keep freed memory in the pool: no release to the driver between requests
        uint64_t keep_all = UINT64_MAX;
        e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
    }
    if (e != cudaSuccess) {
        if (sv->pool) cudaMemPoolDestroy(sv->pool);
        delete sv;
        return server_fail(RSRR_ECUDA, std::string("rsrr_server_create: ") + cudaGetErrorString(e));
    }
    try {
        for (int i = 0; i < sv->o.slots; ++i) sv->workers.emplace_back([sv] { sv->worker(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stopping = true;
        }
        sv->cv_work.notify_all();
        for (auto &t : sv->workers) t.join();
        cudaMemPoolDestroy(sv->pool);
        delete sv;
        return server_fail(RSRR_ENOMEM, "rsrr_server_create: cannot start worker threads");
    }
    *out = reinterpret_cast<rsrr_server_t *>(sv);
    return RSRR_OK;
}

rsrr_status rsrr_server_submit(rsrr_server_t *server, const rsrr_nep *nep, const rsrr_region *region,
                               int32_t N, int32_t L, const rsrr_opts *opts, const rsrr_c128 *U,
                               int64_t *id) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || !id) return server_fail(RSRR_EINVAL, "rsrr_server_submit: server or id is NULL");
    *id = 0;
    const double t_submit = sv->now();
    Handle *h = nullptr;
    rsrr_status st = rsrr::prepare(nep, region, N, L, opts, &h);
    if (st != RSRR_OK) return st;
    if (h->opts.host_threads == 0) {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        h->opts.host_threads = std::max(1, hw / sv->o.slots);
    }
    Request *r = new (std::nothrow) Request();
    if (!r) {
        delete h;
        return server_fail(RSRR_ENOMEM, "rsrr_server_submit: out of host memory");
    }
    r->h = h;
    r->n = h->n;
    r->bytes = h->estimate_bytes();
    r->t_submit = t_submit;
    if (r->bytes > (size_t)sv->o.mem_budget_bytes) {
        char buf[160];
        snprintf(buf, sizeof buf, "rsrr_server_submit: request needs %zu device bytes, budget is %lld",
                 r->bytes, (long long)sv->o.mem_budget_bytes);
        delete h;
        delete r;
        return server_fail(RSRR_ENOMEM, buf);
    }
    if (U) {
        const size_t cnt = (size_t)h->n * h->L;
        r->U.resize(cnt);
        memcpy(r->U.data(), U, sizeof(double2) * cnt);
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) {
            delete h;
            delete r;
            return server_fail(RSRR_ESTATE, "rsrr_server_submit: server is shutting down");
        }
        r->id = sv->next_id++;
        sv->reqs[r->id] = r;
        sv->queue.push_back(r);
        sv->submitted++;
        *id = r->id;
    }
    sv->cv_work.notify_one();
    return RSRR_OK;
}

rsrr_status rsrr_server_wait(rsrr_server_t *server, int64_t id, double timeout_s, rsrr_reply *out) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || !out) return server_fail(RSRR_EINVAL, "rsrr_server_wait: server or out is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return server_fail(RSRR_EINVAL, "rsrr_server_wait: unknown request id");
    Request *r = it->second;
    auto ready = [r] { return r->done; };
    if (timeout_s < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return RSRR_ETIMEOUT;
    }
    memset(out, 0, sizeof *out);
    out->id = r->id;
    out->status = r->status;
    out->count = r->count;
    out->nbar = r->nbar;
    out->k = r->k;
    out->refine_sweeps = r->sweeps;
    out->gmax = r->gmax;
    out->max_eta = r->max_eta;
    out->t_submit = r->t_submit;
    out->t_admit = r->t_admit;
    out->t_done = r->t_done;
    out->t_sample = r->t_sample;
    out->t_project = r->t_project;
    out->t_solve = r->t_solve;
    out->device_bytes = r->bytes;
    out->n = r->n;
    out->lam = r->lam.data();
    out->res = r->res.data();
    out->V = r->V.data();
    out->error = r->error.c_str();
    return RSRR_OK;
}

rsrr_t *rsrr_server_handle(rsrr_server_t *server, int64_t id) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return nullptr;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end() || !it->second->done) return nullptr;
    return reinterpret_cast<rsrr_t *>(it->second->h);
}

rsrr_status rsrr_server_release(rsrr_server_t *server, int64_t id) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return server_fail(RSRR_EINVAL, "rsrr_server_release: server is NULL");
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->reqs.find(id);
        if (it == sv->reqs.end()) return server_fail(RSRR_EINVAL, "rsrr_server_release: unknown request id");
        if (!it->second->done) return server_fail(RSRR_ESTATE, "rsrr_server_release: request not finished");
        r = it->second;
        sv->reqs.erase(it);
    }
    if (r->h) {
        // a kept handle: its device memory goes back to the pool
        cudaSetDevice(sv->device);
        cudaDeviceSynchronize();
        delete r->h;
        cudaDeviceSynchronize();
        r->h = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (r->holds_budget) sv->used -= r->bytes;
    }
    delete r;
    sv->cv_work.notify_all();
    return RSRR_OK;
}

rsrr_status rsrr_server_get_stats(rsrr_server_t *server, rsrr_server_stats *out) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || !out) return server_fail(RSRR_EINVAL, "rsrr_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof *out);
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued = (int32_t)sv->queue.size();
    out->active = sv->active;
    out->peak_active = sv->peak_active;
    out->used_bytes = sv->used;
    out->peak_bytes = sv->peak_used;
    out->budget_bytes = (size_t)sv->o.mem_budget_bytes;
    out->now = sv->now();
    return RSRR_OK;
}

void rsrr_server_destroy(rsrr_server_t *server) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    cudaSetDevice(sv->device);
    cudaDeviceSynchronize();
    for (auto &kv : sv->reqs) {
        delete kv.second->h;
        delete kv.second;
    }
    cudaDeviceSynchronize();
    cudaMemPoolDestroy(sv->pool);
    delete sv;
}

}  // extern "C"
