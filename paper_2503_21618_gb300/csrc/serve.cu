// Many problems at once: a batched entry point and a request server.
//
// Batching: independent pencils are solved concurrently, one handle (and so
// one CUDA stream and one workspace) per problem, each driven by a host
// thread; the problems' kernels overlap on the GPU.  Every kernel reduces in a
// fixed order, so a problem's result in a batch is bit-identical to its result
// alone.
//
// Serving: requests (a host pencil, a pole set, an interval, a start block)
// arrive at any time.  A pool of workers admits them in arrival order as soon
// as the request's device-memory estimate fits in the free part of the
// server's budget, runs Algorithm 1 on a handle of its own (stream-ordered
// allocations on the worker's stream), and files the result for polling.
// Requests that arrive while others run start as soon as a worker and the
// memory are free, so their work overlaps with the running ones on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "slrf.h"

using namespace slrf;

// ---------------------------------------------------------------------------
// batch
// ---------------------------------------------------------------------------
extern "C" slrf_status slrf_batch_iterate(int32_t nprob, slrf_handle *const *h, const slrf_filter *f,
                                          const double *gamma, const int32_t *L, const double *const *V0,
                                          const int64_t *ldv, double tol, int32_t max_outer, double *const *theta,
                                          double *const *X, const int64_t *ldx, double *const *resid,
                                          int32_t *n_conv, slrf_status *status, slrf_report *rep,
                                          int32_t n_threads) {
    if (nprob < 1 || !h || !f || !gamma || !L || !V0 || !ldv || !theta || !X || !ldx || !resid || !n_conv ||
        !status)
        return SLRF_EINVAL;
    for (int i = 0; i < nprob; ++i) {
        if (!h[i]) return SLRF_EINVAL;
        for (int j = 0; j < i; ++j)
            if (h[j] == h[i]) return SLRF_EINVAL;   // each problem needs its own handle (workspace, stream)
    }
    const int nt = n_threads <= 0 ? nprob : std::min<int>(n_threads, nprob);
    std::atomic<int> next{0};
    const char *dbg = getenv("SLRF_DEBUG");
    const bool debug = dbg && dbg[0] && dbg[0] != '0';
    auto work = [&]() {
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nprob) return;
            cudaSetDevice(handle_device(h[i]));
            status[i] = slrf_subspace_iterate(h[i], &f[i], gamma[i], L[i], V0[i], ldv[i], tol, max_outer, theta[i],
                                              X[i], ldx[i], resid[i], &n_conv[i], rep ? &rep[i] : nullptr);
            // the error text is per thread: with SLRF_DEBUG set, report it here
            if (status[i] != SLRF_OK && debug)
                fprintf(stderr, "slrf_batch_iterate: problem %d: %s (%s)\n", i, slrf_status_str(status[i]),
                        slrf_last_error());
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    for (int i = 0; i < nprob; ++i)
        if (status[i] != SLRF_OK) return status[i];
    return SLRF_OK;
}

// ---------------------------------------------------------------------------
// server
// ---------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    int64_t n = 0, nnz = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> av, bv;
    std::vector<double> sre, sim, wre, wim;
    double gamma = 0;
    int32_t L = 0;
    std::vector<double> V0;
    double tol = 1e-8;
    int32_t max_outer = 50;
    slrf_opts opts;
    std::vector<double> nul;   // the options' near-null space (opts points here)
    size_t bytes = 0;
    Clock::time_point t_submit;
};

struct Result {
    bool done = false;
    slrf_status status = SLRF_PENDING;
    std::vector<double> theta, X, resid;
    int32_t n_conv = 0;
    slrf_report rep;
    double latency_ms = 0;
};

}  // namespace

struct slrf_server {
    int device = 0;
    int sm_count = 152;
    size_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_admit, cv_done;
    std::deque<Request *> queue;
    std::map<int64_t, Result *> results;
    std::vector<std::thread> workers;
    bool stop = false;
    int64_t next_ticket = 1;
    int64_t running = 0, finished = 0;
};

namespace {

// Coarsest-size target to budget for when the request's preconditioner may
// resolve to multigrid (AUTO is budgeted as multigrid: an upper bound), else 0.
int request_mg_coarse(const slrf_opts &o) {
    return (o.precond == SLRF_PRECOND_MG || o.precond == SLRF_PRECOND_AUTO) ? o.mg_coarse : 0;
}

void worker_main(slrf_server *s) {
    cudaSetDevice(s->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            // Admit the head of the queue once it fits; a request is accepted
            // only if it fits the whole budget, so with nothing running the
            // head always fits.  On stop, drain the queue, then exit.
            s->cv_admit.wait(lock, [&] {
                return (!s->queue.empty() && s->in_use + s->queue.front()->bytes <= s->budget) ||
                       (s->stop && s->queue.empty());
            });
            if (s->queue.empty()) break;
            r = s->queue.front();
            s->queue.pop_front();
            s->in_use += r->bytes;
            ++s->running;
        }
        Result *res = new Result();
        memset(&res->rep, 0, sizeof(res->rep));
        slrf_pencil p{r->n, r->nnz, r->rp.data(), r->ci.data(), r->av.data(), r->bv.data(), 0};
        slrf_filter f{(int32_t)r->sre.size(), r->sre.data(), r->sim.data(), r->wre.data(), r->wim.data()};
        slrf_handle *h = nullptr;
        res->status = slrf_create(&h, &p, &r->opts, stream);
        if (res->status == SLRF_OK) {
            res->theta.assign(r->L, 0.0);
            res->X.assign((size_t)r->n * r->L, 0.0);
            res->resid.assign(r->L, 0.0);
            res->status = slrf_subspace_iterate_host(h, &f, r->gamma, r->L, r->V0.data(), r->L, r->tol, r->max_outer,
                                                     res->theta.data(), res->X.data(), r->L, res->resid.data(),
                                                     &res->n_conv, &res->rep);
            slrf_destroy(h);
        }
        res->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
        res->done = true;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->in_use -= r->bytes;
            --s->running;
            ++s->finished;
            delete s->results[r->ticket];
            s->results[r->ticket] = res;
        }
        delete r;
        s->cv_admit.notify_all();
        s->cv_done.notify_all();
    }
    cudaStreamDestroy(stream);
}

}  // namespace

extern "C" int64_t slrf_request_bytes(const slrf_request *r) {
    if (!r) return -1;
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    return (int64_t)workspace_estimate(r->pencil.n, r->pencil.nnz, r->L, r->filter.n_poles, r->opts.precision, sms,
                                       request_mg_coarse(r->opts), r->opts.krylov);
}

extern "C" slrf_status slrf_server_create(slrf_server **out, int32_t n_workers, int64_t mem_budget) {
    if (!out || n_workers < 1 || n_workers > 64 || mem_budget < 0) return SLRF_EINVAL;
    *out = nullptr;
    slrf_server *s = new slrf_server();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return SLRF_ECUDA;
    }
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    if (mem_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete s;
            return SLRF_ECUDA;
        }
        s->budget = (size_t)(0.9 * (double)free_b);
    } else {
        s->budget = (size_t)mem_budget;
    }
    for (int i = 0; i < n_workers; ++i) s->workers.emplace_back(worker_main, s);
    *out = s;
    return SLRF_OK;
}

extern "C" slrf_status slrf_server_submit(slrf_server *s, const slrf_request *r, int64_t *ticket) {
    if (!s || !r || !ticket) return SLRF_EINVAL;
    const slrf_pencil &p = r->pencil;
    const slrf_filter &f = r->filter;
    if (p.on_device || p.n < 1 || p.nnz < p.n || !p.row_ptr || !p.col_idx || !p.a_val || !p.b_val || !r->V0 ||
        r->L < 1 || r->L > p.n || f.n_poles < 1 || f.n_poles > SLRF_MAX_POLES || !f.sigma_re || !f.sigma_im ||
        !f.w_re || !f.w_im || !(r->gamma > 0) || !(r->tol > 0) || r->max_outer < 1)
        return SLRF_EINVAL;
    Request *q = new Request();
    q->n = p.n;
    q->nnz = p.nnz;
    q->rp.assign(p.row_ptr, p.row_ptr + p.n + 1);
    q->ci.assign(p.col_idx, p.col_idx + p.nnz);
    q->av.assign(p.a_val, p.a_val + p.nnz);
    q->bv.assign(p.b_val, p.b_val + p.nnz);
    q->sre.assign(f.sigma_re, f.sigma_re + f.n_poles);
    q->sim.assign(f.sigma_im, f.sigma_im + f.n_poles);
    q->wre.assign(f.w_re, f.w_re + f.n_poles);
    q->wim.assign(f.w_im, f.w_im + f.n_poles);
    q->gamma = r->gamma;
    q->L = r->L;
    q->V0.assign(r->V0, r->V0 + (size_t)p.n * r->L);
    q->tol = r->tol;
    q->max_outer = r->max_outer;
    q->opts = r->opts;
    if (r->opts.mg_n_null > 0) {   // copied: the caller's array need not outlive the call
        if (r->opts.mg_n_null > 16 || !r->opts.mg_near_null) {
            delete q;
            return SLRF_EINVAL;
        }
        q->nul.assign(r->opts.mg_near_null, r->opts.mg_near_null + (size_t)p.n * r->opts.mg_n_null);
        q->opts.mg_near_null = q->nul.data();
    } else {
        q->opts.mg_near_null = nullptr;
    }
    q->bytes = workspace_estimate(p.n, p.nnz, r->L, f.n_poles, r->opts.precision, s->sm_count,
                                  request_mg_coarse(r->opts), r->opts.krylov);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (q->bytes > s->budget) {
            delete q;
            return SLRF_EBUDGET;   // could never be admitted
        }
        q->ticket = s->next_ticket++;
        *ticket = q->ticket;
        s->results[q->ticket] = new Result();
        s->queue.push_back(q);
    }
    s->cv_admit.notify_all();
    return SLRF_OK;
}

extern "C" slrf_status slrf_server_poll(slrf_server *s, int64_t ticket, int32_t wait, double *theta, double *X,
                                        double *resid, int32_t *n_conv, slrf_report *rep, double *latency_ms,
                                        slrf_status *result) {
    if (!s) return SLRF_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return SLRF_EINVAL;
    if (!it->second->done) {
        if (!wait) return SLRF_PENDING;
        s->cv_done.wait(lock, [&] { return it->second->done; });
    }
    Result *res = it->second;
    s->results.erase(it);
    lock.unlock();
    if (theta && !res->theta.empty()) std::copy(res->theta.begin(), res->theta.end(), theta);
    if (X && !res->X.empty()) std::copy(res->X.begin(), res->X.end(), X);
    if (resid && !res->resid.empty()) std::copy(res->resid.begin(), res->resid.end(), resid);
    if (n_conv) *n_conv = res->n_conv;
    if (rep) *rep = res->rep;
    if (latency_ms) *latency_ms = res->latency_ms;
    if (result) *result = res->status;
    delete res;
    return SLRF_OK;
}

extern "C" slrf_status slrf_server_stats(slrf_server *s, int64_t *queued, int64_t *running, int64_t *finished,
                                         int64_t *bytes_in_use) {
    if (!s) return SLRF_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = s->running;
    if (finished) *finished = s->finished;
    if (bytes_in_use) *bytes_in_use = (int64_t)s->in_use;
    return SLRF_OK;
}

extern "C" void slrf_server_destroy(slrf_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_admit.notify_all();
    for (auto &t : s->workers) t.join();
    for (Request *q : s->queue) delete q;
    for (auto &kv : s->results) delete kv.second;
    delete s;
}
