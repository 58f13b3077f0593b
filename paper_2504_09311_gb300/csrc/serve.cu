// serve.cu -- continuous batching of peel requests over resident graphs.
//
// A worker thread owns 'max_slots' non-blocking CUDA streams.  Requests wait
// in a queue.  Whenever a slot is free, the worker takes the queued requests
// for graphs small enough for one CTA (as many as the device-memory budget
// admits, in arrival order, passing over large requests that cannot start
// yet) and launches them together as one persistent one-CTA-per-graph peel
// on that slot's stream; it does not wait for it, so requests arriving
// meanwhile go into the next launch on another slot and the launches run side
// by side on the GPU.  A graph that needs the grid-wide persistent kernel
// starts as soon as a slot and the budget allow and no other large request
// is running: on a high-priority stream (its blocks are placed first as SMs
// free up) with a cooperative grid smaller than the GPU by a reserve of SMs,
// so the small requests admitted before and after it keep running beside
// it, and its tail (one CTA or a cluster) runs beside them too.  Graphs stay
// resident and shared; only per-request state is allocated (stream-ordered,
// counted against the budget).  Every request's arithmetic is the same exact
// integer peel, so a result is identical whether it ran alone or in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dupin_internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    dupin_graph *g = nullptr;
    dupin_params p{};
    dupin_result *r = nullptr;
    PeelPlan plan;
    long long bytes = 0;
    bool large = false;
    double t_submit = 0, t_done = 0;
    int status = DUPIN_OK;
    bool done = false;
};

// SMs a running large request leaves to the small requests' launches
#define SERVE_SMALL_RESERVE 32

// what one slot is running: a batch of small requests, or one large request
struct Slot {
    std::vector<Request *> reqs;
    CtaBatch *batch = nullptr;
    PeelWorkspace *ws = nullptr;  // large request
    long long bytes = 0;
    bool busy = false;
    bool large = false;
    cudaStream_t st = nullptr;  // the stream its work runs on
    cudaEvent_t ev = nullptr;   // recorded after it
    // the batch entry point wants arrays indexed by position
    std::vector<dupin_graph *> gs;
    std::vector<dupin_params> ps;
    std::vector<dupin_result> rs;
};

}  // namespace

struct dupin_server {
    dupin_serve_config cfg{};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable done_cv;  // wakes waiters
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<Slot> slots;
    cudaStream_t large_stream = nullptr;  // high priority, for the one running large request
    cudaEvent_t large_event = nullptr;
    long long used_bytes = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool large_running = false;
    long long submitted = 0, completed = 0, rejected = 0, launches = 0;
    std::vector<double> lat_ms;
    double first_submit = -1, last_done = 0;
};

static int n_busy(const dupin_server *s) {
    int k = 0;
    for (const auto &sl : s->slots) k += sl.busy ? 1 : 0;
    return k;
}

static const size_t kMaxBatch = 4096;

// Fill free slots from the queue (lock held on entry and exit).
static bool admit(dupin_server *s, std::unique_lock<std::mutex> &lk) {
    bool progress = false;
    for (;;) {
        if (s->queue.empty()) return progress;
        int slot = -1;
        for (int i = 0; i < (int)s->slots.size(); i++)
            if (!s->slots[i].busy) {
                slot = i;
                break;
            }
        if (slot < 0) return progress;
        Slot &sl = s->slots[slot];
        sl.reqs.clear();
        sl.bytes = 0;
        // the first large request in arrival order starts once none is running
        // and the budget admits it
        Request *big = nullptr;
        if (!s->large_running) {
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                if (!(*it)->large) continue;
                if (s->used_bytes + (*it)->bytes <= s->cfg.memory_budget) {
                    big = *it;
                    s->queue.erase(it);
                }
                break;
            }
        }
        if (big) {
            sl.reqs.push_back(big);
            sl.bytes = big->bytes;
            sl.large = true;
            sl.st = s->large_stream;
            sl.ev = s->large_event;
            s->large_running = true;
        } else {
            // small requests in arrival order (large ones that cannot start are
            // passed over), within the budget
            for (auto it = s->queue.begin(); it != s->queue.end() && sl.reqs.size() < kMaxBatch;) {
                Request *q = *it;
                if (q->large) {
                    ++it;
                    continue;
                }
                if (s->used_bytes + sl.bytes + q->bytes > s->cfg.memory_budget) break;
                it = s->queue.erase(it);
                sl.reqs.push_back(q);
                sl.bytes += q->bytes;
            }
            if (sl.reqs.empty()) return progress;
            sl.large = false;
            sl.st = s->streams[slot];
            sl.ev = s->events[slot];
        }
        s->used_bytes += sl.bytes;
        sl.busy = true;
        s->launches++;
        lk.unlock();
        cudaStream_t st = sl.st;
        int rc = DUPIN_OK;
        if (sl.large) {
            Request *q = sl.reqs[0];
            sl.ws = workspace_create(q->g->n, q->g->arcs, q->g->cw != nullptr, q->plan, true, st, &rc);
            if (rc == DUPIN_OK) {
                const int grid = sl.ws->grid - SERVE_SMALL_RESERVE;
                rc = enqueue_peel_stages(q->g, sl.ws, &q->p, q->plan, PEEL_ALL, st, nullptr, grid > 16 ? grid : 16);
            }
        } else {
            const size_t k = sl.reqs.size();
            sl.gs.resize(k);
            sl.ps.resize(k);
            sl.rs.resize(k);
            std::vector<int64_t> idx(k);
            for (size_t j = 0; j < k; j++) {
                sl.gs[j] = sl.reqs[j]->g;
                sl.ps[j] = sl.reqs[j]->p;
                sl.rs[j] = *sl.reqs[j]->r;
                idx[j] = (int64_t)j;
            }
            rc = cta_batch_enqueue(sl.gs.data(), sl.ps.data(), sl.rs.data(), idx, st, &sl.batch);
        }
        if (rc == DUPIN_OK) {
            cudaError_t e = cudaEventRecord(sl.ev, st);
            if (e != cudaSuccess) rc = dupin_cuda_fail(e, "cudaEventRecord");
        }
        lk.lock();
        if (rc != DUPIN_OK)
            for (Request *q : sl.reqs) q->status = rc;
        progress = true;
    }
}

static void finish_slot(dupin_server *s, int i) {
    Slot &sl = s->slots[i];
    cudaStream_t st = sl.st;
    const bool launched_ok = sl.reqs.empty() || sl.reqs[0]->status == DUPIN_OK;
    if (sl.large) {
        Request *q = sl.reqs[0];
        if (launched_ok) q->status = peel_finish(q->g, sl.ws, &q->p, q->r, st);
        workspace_free(sl.ws, st);
        sl.ws = nullptr;
    } else if (sl.batch) {
        std::vector<int> st_each;
        cta_batch_finish(sl.batch, st, &st_each);
        sl.batch = nullptr;
        for (size_t j = 0; j < sl.reqs.size(); j++) {
            *sl.reqs[j]->r = sl.rs[j];
            if (j < st_each.size() && st_each[j] != DUPIN_OK) sl.reqs[j]->status = st_each[j];
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    for (Request *q : sl.reqs) {
        q->t_done = t;
        q->done = true;
        s->completed++;
        if (q->status == DUPIN_OK) s->lat_ms.push_back((q->t_done - q->t_submit) * 1e3);
    }
    s->last_done = t;
    s->used_bytes -= sl.bytes;
    if (sl.large) s->large_running = false;
    sl.busy = false;
    sl.reqs.clear();
    s->done_cv.notify_all();
}

static void serve_loop(dupin_server *s) {
    cudaSetDevice(s->cfg.device);
    for (;;) {
        bool progress = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->queue.empty() && n_busy(s) == 0) break;
            progress = admit(s, lk);
        }
        for (int i = 0; i < (int)s->slots.size(); i++) {
            bool busy;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                busy = s->slots[i].busy;
            }
            if (!busy) continue;
            const bool failed = !s->slots[i].reqs.empty() && s->slots[i].reqs[0]->status != DUPIN_OK;
            if (!failed) {
                cudaError_t e = cudaEventQuery(s->slots[i].ev);
                if (e == cudaErrorNotReady) continue;
                if (e != cudaSuccess) {
                    const int rc = dupin_cuda_fail(e, "request kernels");
                    for (Request *q : s->slots[i].reqs) q->status = rc;
                }
            }
            finish_slot(s, i);
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (n_busy(s) > 0) {
                lk.unlock();
                std::this_thread::yield();
            } else {
                s->cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return s->stop || !s->queue.empty(); });
            }
        }
    }
}

extern "C" int dupin_serve_create(const dupin_serve_config *cfg, dupin_server **out) {
    if (!cfg || !out) return dupin_fail(DUPIN_ERR_INVALID_ARG, "cfg or out is NULL");
    if (cfg->memory_budget <= 0 || cfg->max_slots < 1 || cfg->max_slots > 4096)
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "memory_budget > 0 and 1 <= max_slots <= 4096 required");
    DUPIN_CUDA_TRY(cudaSetDevice(cfg->device));
    dupin_server *s = new dupin_server();
    s->cfg = *cfg;
    s->streams.resize(cfg->max_slots);
    s->events.resize(cfg->max_slots);
    s->slots.resize(cfg->max_slots);
    {
        int lo = 0, hi = 0;  // numerically lower is higher priority
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->large_stream, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->large_event, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (s->large_stream) cudaStreamDestroy(s->large_stream);
            delete s;
            return dupin_cuda_fail(e, "serving stream for large requests");
        }
    }
    for (int i = 0; i < cfg->max_slots; i++) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; j++) {
                cudaStreamDestroy(s->streams[j]);
                cudaEventDestroy(s->events[j]);
            }
            cudaStreamDestroy(s->large_stream);
            cudaEventDestroy(s->large_event);
            delete s;
            return dupin_cuda_fail(e, "serving streams");
        }
    }
    s->worker = std::thread(serve_loop, s);
    *out = s;
    return DUPIN_OK;
}

extern "C" int dupin_serve_submit(dupin_server *s, dupin_graph *g, const dupin_params *p, dupin_result *r,
                                  uint64_t *ticket) {
    if (!s || !g || !p || !r || !ticket) return dupin_fail(DUPIN_ERR_INVALID_ARG, "NULL argument");
    Request *q = new Request();
    q->g = g;
    q->p = *p;
    q->r = r;
    int rc = peel_resolve(g, p, &q->plan);
    if (rc == DUPIN_OK && is_clique_metric(p->metric))
        rc = dupin_fail(DUPIN_ERR_INVALID_ARG, "the clique metrics (TDS, kCLiDS) are served by dupin_peel only");
    if (rc) {
        delete q;
        return rc;
    }
    if (p->flags & DUPIN_RESULT_DEVICE) {
        delete q;
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "serving writes host results; DUPIN_RESULT_DEVICE is not accepted");
    }
    q->large = g->n < 1 || g->n > cta_graph_limit();
    q->bytes = q->large ? workspace_bytes(g->n, g->arcs, g->cw != nullptr, q->plan, peel_grid_size())
                        : cta_job_bytes(g, p);
    q->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    *ticket = q->ticket;
    s->submitted++;
    if (s->first_submit < 0) s->first_submit = q->t_submit;
    if (q->bytes > s->cfg.memory_budget) {
        s->rejected++;
        q->status = DUPIN_ERR_OOM;
        q->done = true;
        q->t_done = q->t_submit;
        s->all[q->ticket] = q;
        return dupin_fail(DUPIN_ERR_OOM, "request state exceeds the whole serving memory budget");
    }
    s->all[q->ticket] = q;
    s->queue.push_back(q);
    s->cv.notify_all();
    return DUPIN_OK;
}

extern "C" int dupin_serve_poll(dupin_server *s, uint64_t ticket, int *done, int *status) {
    if (!s || !done) return dupin_fail(DUPIN_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return dupin_fail(DUPIN_ERR_NOT_FOUND, "unknown ticket");
    *done = it->second->done ? 1 : 0;
    if (status) *status = it->second->status;
    return DUPIN_OK;
}

extern "C" int dupin_serve_wait(dupin_server *s, uint64_t ticket, int *status) {
    if (!s) return dupin_fail(DUPIN_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return dupin_fail(DUPIN_ERR_NOT_FOUND, "unknown ticket");
    Request *q = it->second;
    s->done_cv.wait(lk, [&] { return q->done; });
    if (status) *status = q->status;
    s->all.erase(it);
    delete q;
    return DUPIN_OK;
}

extern "C" int dupin_serve_stats(dupin_server *s, dupin_serve_stats_t *out) {
    if (!s || !out) return dupin_fail(DUPIN_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->in_flight = 0;
    for (const auto &sl : s->slots) out->in_flight += sl.busy ? (int64_t)sl.reqs.size() : 0;
    out->queued = (int64_t)s->queue.size();
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        size_t k = (size_t)std::min<double>((double)v.size() - 1, q * (double)v.size());
        return v[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double span = s->last_done - s->first_submit;
    out->graphs_per_s = (s->completed > 0 && span > 0) ? (double)s->completed / span : 0.0;
    return DUPIN_OK;
}

extern "C" int dupin_serve_destroy(dupin_server *s) {
    if (!s) return DUPIN_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->all) delete kv.second;
    for (size_t i = 0; i < s->streams.size(); i++) {
        cudaStreamDestroy(s->streams[i]);
        cudaEventDestroy(s->events[i]);
    }
    cudaStreamDestroy(s->large_stream);
    cudaEventDestroy(s->large_event);
    delete s;
    return DUPIN_OK;
}
