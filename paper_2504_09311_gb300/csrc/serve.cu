// serve.cu -- continuous batching of peel requests over resident graphs.
//
// A worker thread owns 'max_slots' non-blocking CUDA streams.  Requests wait
// in a FIFO queue and are admitted into a free slot as soon as the
// device-memory budget has room for their per-request state (a peeling
// workspace allocated stream-ordered on the slot's stream); graphs
// themselves stay resident and are shared.  Admitted requests run
// concurrently -- a graph small enough for the one-CTA peel occupies one SM,
// so many of them overlap -- while new requests keep being admitted as
// earlier ones finish.  A graph that needs the grid-wide persistent kernel
// runs alone (it is admitted only when no other slot is busy and nothing is
// admitted beside it), so co-residency of its cooperative grid is never in
// question.  Every request's arithmetic is the same exact integer peel, so a
// result is identical whether it ran alone or in a mix.
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
    long long tail_cap = 0, max_rounds = 0, tr_cap = 0, bytes = 0;
    bool large = false;
    double t_submit = 0, t_done = 0;
    int status = DUPIN_OK;
    bool done = false;
    PeelWorkspace *ws = nullptr;
    int slot = -1;
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
    std::vector<Request *> running;
    long long used_bytes = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool exclusive = false;
    long long submitted = 0, completed = 0, rejected = 0;
    std::vector<double> lat_ms;
    double first_submit = -1, last_done = 0;
};

static int n_running(const dupin_server *s) {
    int k = 0;
    for (auto *q : s->running) k += q != nullptr;
    return k;
}

static void serve_loop(dupin_server *s) {
    cudaSetDevice(s->cfg.device);
    for (;;) {
        bool progress = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->queue.empty() && n_running(s) == 0) break;
            // admission, first come first served
            while (!s->queue.empty()) {
                Request *q = s->queue.front();
                const int busy = n_running(s);
                if (s->exclusive) break;
                if (q->large && busy > 0) break;
                int slot = -1;
                for (int i = 0; i < (int)s->running.size(); i++)
                    if (!s->running[i]) {
                        slot = i;
                        break;
                    }
                if (slot < 0) break;
                if (s->used_bytes + q->bytes > s->cfg.memory_budget) break;
                s->queue.pop_front();
                s->used_bytes += q->bytes;
                q->slot = slot;
                s->running[slot] = q;
                if (q->large) s->exclusive = true;
                lk.unlock();
                cudaStream_t st = s->streams[slot];
                int rc = DUPIN_OK;
                q->ws = workspace_create(q->g->n, q->g->arcs, q->g->cw != nullptr, q->tail_cap, q->tr_cap, true, st, &rc);
                if (rc == DUPIN_OK) rc = enqueue_peel(q->g, q->ws, &q->p, q->tail_cap, q->max_rounds, st);
                if (rc == DUPIN_OK) {
                    cudaError_t e = cudaEventRecord(s->events[slot], st);
                    if (e != cudaSuccess) rc = dupin_cuda_fail(e, "cudaEventRecord");
                }
                lk.lock();
                if (rc != DUPIN_OK) {
                    q->status = rc;
                    q->ws = q->ws;  // freed below with the others
                }
                progress = true;
            }
        }
        // completions
        for (int i = 0; i < (int)s->running.size(); i++) {
            Request *q;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                q = s->running[i];
            }
            if (!q) continue;
            if (q->status == DUPIN_OK) {
                cudaError_t e = cudaEventQuery(s->events[i]);
                if (e == cudaErrorNotReady) continue;
                if (e != cudaSuccess) q->status = dupin_cuda_fail(e, "request kernels");
                else q->status = peel_finish(q->g, q->ws, &q->p, q->r, s->streams[i]);
            }
            workspace_free(q->ws, s->streams[i]);
            q->ws = nullptr;
            std::lock_guard<std::mutex> lk(s->mu);
            q->t_done = now_s();
            q->done = true;
            s->running[i] = nullptr;
            s->used_bytes -= q->bytes;
            if (q->large) s->exclusive = false;
            s->completed++;
            if (q->status == DUPIN_OK) s->lat_ms.push_back((q->t_done - q->t_submit) * 1e3);
            s->last_done = q->t_done;
            s->done_cv.notify_all();
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (n_running(s) > 0) {
                lk.unlock();
                std::this_thread::yield();
            } else {
                s->cv.wait_for(lk, std::chrono::milliseconds(2),
                               [&] { return s->stop || !s->queue.empty(); });
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
    s->running.assign(cfg->max_slots, nullptr);
    for (int i = 0; i < cfg->max_slots; i++) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; j++) {
                cudaStreamDestroy(s->streams[j]);
                cudaEventDestroy(s->events[j]);
            }
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
    int rc = peel_resolve(g, p, &q->tail_cap, &q->max_rounds, &q->tr_cap);
    if (rc) {
        delete q;
        return rc;
    }
    if (p->flags & DUPIN_RESULT_DEVICE) {
        delete q;
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "serving writes host results; DUPIN_RESULT_DEVICE is not accepted");
    }
    q->large = g->n > q->tail_cap;
    q->bytes = workspace_bytes(g->n, g->arcs, g->cw != nullptr, q->tail_cap, q->tr_cap, peel_grid_size());
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
    out->in_flight = n_running(s);
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
    delete s;
    return DUPIN_OK;
}
