// Continuous-batching serving loop for GA inversions (host C++ runtime).
//
// Requests (slit scans, map tiles of any pixel count) are copied on submit
// and queued.  A worker thread admits them in arrival order whenever an
// in-flight slot is free and their buffers fit the arena (admission by
// memory), stages them through a pinned host arena into a device arena, and
// launches the GA (and optionally the L-M polish) on a stream of their own, so
// admitted requests overlap on the device: their thread blocks interleave on
// the SMs as earlier requests drain.  Completion is detected with events; the
// results are copied out and the arena range is released for the next
// request.  Each request's kernels see only its own pixels and its own pixel
// ids, so a result is bit-identical whether it ran alone or in a mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "genesis.h"
#include "kernels.h"

struct serve_handle;

namespace genesis {

namespace {

using Clock = std::chrono::steady_clock;

uint64_t ns_since(Clock::time_point t0, Clock::time_point t1)
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(t1 - t0).count();
}

enum class State { Queued, Running, Done };

struct Layout {
    size_t obs, w, mu, pw, best, chi2, total;
};

Layout layout_for(int npix, int n_lambda, int npar, size_t elem, bool has_w, bool has_mu, bool has_pw)
{
    Layout L;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        const size_t off = at;
        at = Arena::round_up(at + bytes, 256);
        return off;
    };
    L.obs = take((size_t)npix * 4 * n_lambda * elem);
    L.w = has_w ? take((size_t)npix * 4 * 8) : 0;
    L.mu = has_mu ? take((size_t)npix * 8) : 0;
    L.pw = has_pw ? take((size_t)npix * 4 * 8) : 0;
    L.best = take((size_t)npix * npar * 8);
    L.chi2 = take((size_t)npix * 8);
    L.total = at;
    return L;
}

struct Request {
    uint64_t ticket = 0;
    serve_request rq{};
    std::vector<unsigned char> obs;
    std::vector<double> w, mu, pw;
    Layout lay{};
    size_t off = Arena::kNone;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    State state = State::Queued;
    int status = ME_OK;
    Clock::time_point t_submit, t_admit, t_done;
    bool admitted = false;
    std::vector<double> best, chi2;
};

}  // namespace
}  // namespace genesis

using namespace genesis;

struct serve_handle {
    int device = 0;
    me_problem pb{};
    std::vector<double> lambda;
    KProblem kp{};
    serve_config cfg{};
    size_t elem = 4;
    void *d_arena = nullptr;
    unsigned char *h_arena = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<cudaStream_t> free_lo, free_hi;
    std::vector<cudaEvent_t> free_ev;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    int fail_admissions = 0;
};

namespace {

// Enqueue one admitted request's copies and kernels on its stream.
int launch_request(serve_handle *h, Request *r)
{
    const serve_request &q = r->rq;
    unsigned char *hb = h->h_arena + r->off;
    unsigned char *db = (unsigned char *)h->d_arena + r->off;
    const Layout &L = r->lay;
    std::memcpy(hb + L.obs, r->obs.data(), r->obs.size());
    if (!r->w.empty()) std::memcpy(hb + L.w, r->w.data(), r->w.size() * 8);
    if (!r->mu.empty()) std::memcpy(hb + L.mu, r->mu.data(), r->mu.size() * 8);
    if (!r->pw.empty()) std::memcpy(hb + L.pw, r->pw.data(), r->pw.size() * 8);
    cudaStream_t st = r->stream;
    cudaError_t e = cudaMemcpyAsync(db, hb, L.best, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "serve H2D");
    KGa g;
    const int npar = npar_of(&h->pb);
    int rc = make_ga(&q.ga, &q.bounds, q.pixel_id0, g, npar);
    if (rc) return rc;
    const double *dw = r->w.empty() ? nullptr : (const double *)(db + L.w);
    const double *dmu = r->mu.empty() ? nullptr : (const double *)(db + L.mu);
    const double *dpw = r->pw.empty() ? dw : (const double *)(db + L.pw);
    double *dbest = (double *)(db + L.best);
    double *dchi2 = (double *)(db + L.chi2);
    e = launch_ga_evolve(h->kp, g, h->pb.dtype, db + L.obs, q.ga.weight_mode == ME_W_USER ? dw : nullptr,
                         dmu, q.npix, dbest, nullptr, st);
    if (e != cudaSuccess) return cuda_error(e, "serve GA launch");
    if (q.polish_iters > 0) {
        KLm lm;
        std::memset(&lm, 0, sizeof lm);
        lm.iters = q.polish_iters;
        lm.lambda0 = q.lambda0;
        lm.free_mask = (1u << npar) - 1u;
        for (int d = 0; d < npar; ++d) {
            lm.lo[d] = q.bounds.lo[d];
            lm.hi[d] = q.bounds.hi[d];
        }
        e = launch_lm(h->kp, lm, h->pb.dtype, db + L.obs, dpw, dmu, q.npix, dbest, st);
        if (e != cudaSuccess) return cuda_error(e, "serve L-M launch");
        e = launch_chi2_f64(h->kp, h->pb.dtype, db + L.obs, dpw, dmu, q.npix, dbest, dchi2, st);
    } else {
        e = launch_chi2_f64(h->kp, h->pb.dtype, db + L.obs,
                            q.ga.weight_mode == ME_W_USER ? dw : nullptr, dmu, q.npix, dbest, dchi2, st);
    }
    if (e != cudaSuccess) return cuda_error(e, "serve chi2 launch");
    e = cudaMemcpyAsync(hb + L.best, db + L.best, L.total - L.best, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "serve D2H");
    e = cudaEventRecord(r->done, st);
    if (e != cudaSuccess) return cuda_error(e, "serve event");
    return ME_OK;
}

void finish(serve_handle *h, Request *r, int status)
{
    r->status = status;
    r->t_done = Clock::now();
    if (r->off != Arena::kNone) {
        if (status == ME_OK) {
            const unsigned char *hb = h->h_arena + r->off;
            r->best.assign((const double *)(hb + r->lay.best),
                           (const double *)(hb + r->lay.best) + (size_t)r->rq.npix * npar_of(&h->pb));
            r->chi2.assign((const double *)(hb + r->lay.chi2),
                           (const double *)(hb + r->lay.chi2) + r->rq.npix);
        }
        h->arena.release(r->off);
        r->off = Arena::kNone;
    }
    if (r->stream) {
        (r->rq.npix <= h->cfg.small_pixels ? h->free_hi : h->free_lo).push_back(r->stream);
        r->stream = nullptr;
    }
    if (r->done) {
        h->free_ev.push_back(r->done);
        r->done = nullptr;
    }
    r->obs.clear();
    r->obs.shrink_to_fit();
    r->state = State::Done;
}

void worker_loop(serve_handle *h)
{
    cudaSetDevice(h->device);
    std::unique_lock<std::mutex> lk(h->mu);
    while (true) {
        // retire finished requests
        bool progressed = false;
        for (size_t i = 0; i < h->running.size();) {
            Request *r = h->running[i];
            const cudaError_t q = cudaEventQuery(r->done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            finish(h, r, q == cudaSuccess ? ME_OK : ME_ECUDA);
            h->running.erase(h->running.begin() + i);
            progressed = true;
        }
        if (progressed) h->cv_done.notify_all();
        if (h->stop && h->running.empty()) break;
        // admit in arrival order while a slot and arena room are free
        while (!h->stop && !h->queue.empty() && (int)h->running.size() < h->cfg.max_inflight) {
            Request *r = h->queue.front();
            if (h->fail_admissions > 0) {
                --h->fail_admissions;
                h->queue.pop_front();
                finish(h, r, ME_ENOMEM);
                h->cv_done.notify_all();
                continue;
            }
            const size_t off = h->arena.alloc(r->lay.total);
            if (off == Arena::kNone) break;  // wait for a running request to free memory
            h->queue.pop_front();
            r->off = off;
            auto &pool = r->rq.npix <= h->cfg.small_pixels ? h->free_hi : h->free_lo;
            r->stream = pool.back();
            pool.pop_back();
            r->done = h->free_ev.back();
            h->free_ev.pop_back();
            r->t_admit = Clock::now();
            r->admitted = true;
            r->state = State::Running;
            const int rc = launch_request(h, r);
            if (rc != ME_OK) {
                cudaStreamSynchronize(r->stream);
                finish(h, r, rc);
                h->cv_done.notify_all();
                continue;
            }
            h->running.push_back(r);
        }
        if (h->stop && h->running.empty()) break;
        if (h->running.empty() && h->queue.empty()) {
            h->cv_work.wait(lk);
        } else {
            h->cv_work.wait_for(lk, std::chrono::microseconds(100));
        }
    }
}

}  // namespace

extern "C" {

int serve_create(const me_problem *pb, const serve_config *cfg, serve_handle **out)
{
    if (!out) return set_error(ME_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return set_error(ME_EINVAL, "serve_config is NULL");
    KProblem kp;
    int rc = make_problem(pb, kp);
    if (rc) return rc;
    if (cfg->arena_bytes < 4096) return set_error(ME_EINVAL, "arena_bytes must be >= 4096");
    if (cfg->max_inflight < 1 || cfg->max_inflight > 64)
        return set_error(ME_EINVAL, "max_inflight must be 1..64");
    if (cfg->max_queue < 1) return set_error(ME_EINVAL, "max_queue must be >= 1");
    if ((rc = ensure_device())) return rc;
    serve_handle *h = new (std::nothrow) serve_handle();
    if (!h) return set_error(ME_ENOMEM, "serve handle allocation failed");
    cudaGetDevice(&h->device);
    h->pb = *pb;
    h->lambda.assign(pb->lambda_A, pb->lambda_A + pb->n_lambda);
    h->pb.lambda_A = h->lambda.data();
    h->kp = kp;
    h->cfg = *cfg;
    h->elem = pb->dtype == ME_F32 ? 4 : 8;
    h->fail_admissions = cfg->fail_next_admissions;
    cudaError_t e = cudaMalloc(&h->d_arena, cfg->arena_bytes);
    if (e != cudaSuccess) {
        delete h;
        cudaGetLastError();
        return set_error(ME_ENOMEM, "device arena allocation failed");
    }
    e = cudaHostAlloc((void **)&h->h_arena, cfg->arena_bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaFree(h->d_arena);
        delete h;
        cudaGetLastError();
        return set_error(ME_ENOMEM, "pinned host arena allocation failed");
    }
    h->arena = Arena(cfg->arena_bytes, 256);
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int i = 0; i < cfg->max_inflight; ++i) {
        cudaStream_t a, b;
        cudaEvent_t ev;
        cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, lo);
        cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, hi);
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        h->free_lo.push_back(a);
        h->free_hi.push_back(b);
        h->free_ev.push_back(ev);
    }
    h->worker = std::thread(worker_loop, h);
    *out = h;
    return ME_OK;
}

int serve_submit(serve_handle *h, const serve_request *rq, uint64_t *ticket)
{
    if (!h || !rq || !ticket) return set_error(ME_EINVAL, "NULL argument");
    if (rq->npix < 1) return set_error(ME_EINVAL, "npix must be >= 1");
    if (!rq->obs) return set_error(ME_EINVAL, "obs is NULL");
    const int npar = npar_of(&h->pb);
    int rc = check_bounds(&rq->bounds, npar);
    if (rc) return rc;
    KGa g;
    if ((rc = make_ga(&rq->ga, &rq->bounds, rq->pixel_id0, g, npar))) return rc;
    if (rq->ga.weight_mode == ME_W_USER && !rq->w) return set_error(ME_EINVAL, "ME_W_USER needs w");
    if (rq->polish_iters < 0) return set_error(ME_EINVAL, "polish_iters must be >= 0");
    if (rq->polish_iters > 0 && !(rq->lambda0 > 0.0)) return set_error(ME_EINVAL, "lambda0 must be > 0");
    if (rq->pixel_id0 + (uint64_t)rq->npix < rq->pixel_id0) return set_error(ME_EINVAL, "pixel id overflow");
    const Layout lay = layout_for(rq->npix, h->pb.n_lambda, npar, h->elem, rq->w != nullptr,
                                  rq->mu_px != nullptr, rq->polish_w != nullptr);
    if (lay.total > h->arena.size()) return set_error(ME_EINVAL, "request larger than the serving arena");
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(ME_ENOMEM, "request allocation failed");
    r->rq = *rq;
    r->lay = lay;
    const size_t nobs = (size_t)rq->npix * 4 * h->pb.n_lambda * h->elem;
    try {
        r->obs.assign((const unsigned char *)rq->obs, (const unsigned char *)rq->obs + nobs);
        if (rq->w) r->w.assign(rq->w, rq->w + (size_t)rq->npix * 4);
        if (rq->mu_px) r->mu.assign(rq->mu_px, rq->mu_px + rq->npix);
        if (rq->polish_w) r->pw.assign(rq->polish_w, rq->polish_w + (size_t)rq->npix * 4);
    } catch (...) {
        delete r;
        return set_error(ME_ENOMEM, "request copy failed");
    }
    r->rq.obs = nullptr;
    r->rq.w = r->rq.mu_px = r->rq.polish_w = nullptr;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(h->mu);
        if (h->stop) {
            delete r;
            return set_error(ME_EINVAL, "serve handle is shutting down");
        }
        if ((int)h->queue.size() >= h->cfg.max_queue) {
            delete r;
            return set_error(ME_EAGAIN, "serve queue full");
        }
        r->ticket = h->next_ticket++;
        h->all[r->ticket] = r;
        h->queue.push_back(r);
        *ticket = r->ticket;
    }
    h->cv_work.notify_one();
    return ME_OK;
}

int serve_poll(serve_handle *h, uint64_t ticket, serve_result *out, int timeout_ms)
{
    if (!h) return set_error(ME_EINVAL, "handle is NULL");
    std::unique_lock<std::mutex> lk(h->mu);
    auto it = h->all.find(ticket);
    if (it == h->all.end()) return set_error(ME_ENOTFOUND, "unknown ticket");
    Request *r = it->second;
    if (r->state != State::Done) {
        if (timeout_ms == 0) return set_error(ME_EPENDING, "request pending");
        auto pred = [&] { return r->state == State::Done; };
        if (timeout_ms < 0) {
            h->cv_done.wait(lk, pred);
        } else if (!h->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
            return set_error(ME_ETIMEOUT, "request still running at the timeout");
        }
    }
    if (out) {
        out->status = r->status;
        out->queue_ns = r->admitted ? ns_since(r->t_submit, r->t_admit) : 0;
        out->latency_ns = ns_since(r->t_submit, r->t_done);
        if (r->status == ME_OK) {
            if (out->best) std::memcpy(out->best, r->best.data(), r->best.size() * 8);
            if (out->chi2) std::memcpy(out->chi2, r->chi2.data(), r->chi2.size() * 8);
        }
    }
    const int status = r->status;
    h->all.erase(it);
    delete r;
    if (status != ME_OK) return set_error(status, "request failed");
    return ME_OK;
}

int serve_stats(serve_handle *h, serve_stats_t *out)
{
    if (!h || !out) return set_error(ME_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(h->mu);
    out->queued = (int)h->queue.size();
    out->running = (int)h->running.size();
    out->arena_used = h->arena.used();
    out->arena_bytes = h->arena.size();
    return ME_OK;
}

int serve_destroy(serve_handle *h)
{
    if (!h) return set_error(ME_EINVAL, "handle is NULL");
    {
        std::lock_guard<std::mutex> lk(h->mu);
        h->stop = true;
        for (Request *r : h->queue) {
            r->status = ME_EINVAL;
            r->state = State::Done;
        }
        h->queue.clear();
    }
    h->cv_work.notify_all();
    h->worker.join();
    for (auto &kv : h->all) delete kv.second;
    h->all.clear();
    for (auto s : h->free_lo) cudaStreamDestroy(s);
    for (auto s : h->free_hi) cudaStreamDestroy(s);
    for (auto e : h->free_ev) cudaEventDestroy(e);
    cudaFree(h->d_arena);
    cudaFreeHost(h->h_arena);
    delete h;
    return ME_OK;
}

}  // extern "C"
