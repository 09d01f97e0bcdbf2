// Serving loop: continuous batching of influence-maximization queries over
// resident graphs and RR pools.
//
// Queries (graph, model, k, eps, ell, seed, options) arrive through hbx_submit
// at any time.  Worker threads (max_inflight of them) take the oldest queued
// query whose pool is free and whose projected device footprint fits the memory
// budget, and run IMM on it.  Pools are kept resident and keyed by (graph,
// model, seed, epoch, encoding options, scheme): a later query on the same key reuses
// the sets already sampled (set j depends only on (seed, epoch, j)) and extends
// them as needed.  Every pool has its own CUDA stream, so queries on different
// pools overlap on the device.  Results equal hbx_imm's for the same arguments.
//
// Admission: a query's projected footprint is its pool's bytes per set (64 B
// before anything is known) times its projected theta, max(current size,
// ceil(lambda* / max(k, last LB seen on that pool))) -- LB >= k holds for any
// seed set of size k, since every seed covers its own sets.  A query whose
// projection exceeds the whole budget is rejected at submission; otherwise it
// waits until resident pools leave room, idle pools being evicted oldest first.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "runtime.h"

using namespace hbx;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum QState { Q_QUEUED, Q_RUNNING, Q_DONE, Q_CANCELLED };

struct Query {
    hbx_graph* g;
    hbx_model model;
    uint32_t k;
    double eps, ell;
    uint64_t seed;
    hbx_options o;
    QState state = Q_QUEUED;
    int rc = 0;
    std::vector<uint32_t> seeds;
    double influence = 0;
    hbx_stats stats{};
    double t_submit = 0, t_done = 0;
    uint64_t projected = 0;
    std::string error;  // message of a failed query
};

using PoolKey = std::tuple<const hbx_graph*, int, uint64_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t>;

struct PoolEntry {
    hbx_pool* pool = nullptr;
    bool busy = false;
    double last_used = 0;
    double last_lb = 0;
};

PoolKey key_of(const Query& q) {
    return PoolKey(q.g, (int)q.model, q.seed, q.o.pool_epoch, q.o.encode, q.o.density_cut, q.o.warmup_sets,
                   q.o.scheme);
}

}  // namespace

struct hbx_server {
    hbx_ctx* ctx = nullptr;
    uint32_t max_inflight = 1;
    uint64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // workers wait for runnable queries
    std::condition_variable cv_done;  // waiters wait for results
    std::deque<std::shared_ptr<Query>> queue;
    std::map<PoolKey, PoolEntry> pools;
    std::vector<std::thread> workers;
    bool stop = false;
};

struct hbx_ticket {
    hbx_server* s = nullptr;
    std::shared_ptr<Query> q;
};

namespace {

uint64_t pool_bytes(const PoolEntry& e) { return e.pool ? e.pool->device_bytes : 0; }

uint64_t project(hbx_server* s, Query& q) {
    double lp = 0, ls = 0;
    if (!imm_lambda(q.g->n, q.k, q.eps, q.ell, &lp, &ls)) return 0;
    auto it = s->pools.find(key_of(q));
    double per_set = 64.0;
    uint64_t have = 0;
    double lb = (double)q.k;
    if (it != s->pools.end() && it->second.pool) {
        const hbx_pool* p = it->second.pool;
        have = p->T;
        if (p->T) per_set = (double)p->device_bytes / (double)p->T;
        lb = std::max(lb, it->second.last_lb);
    }
    const double theta = std::max((double)have, std::ceil(ls / lb));
    return (uint64_t)(per_set * theta) + (uint64_t)q.g->n * 16;  // + selection state
}

uint64_t resident_bytes(hbx_server* s) {
    uint64_t b = 0;
    for (auto& kv : s->pools) b += pool_bytes(kv.second);
    return b;
}

// Pick the oldest queued query that can run now (its pool is idle and its
// projection fits after evicting idle pools); called with s->mu held.
std::shared_ptr<Query> pick(hbx_server* s) {
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Query& q = **it;
        auto pe = s->pools.find(key_of(q));
        if (pe != s->pools.end() && pe->second.busy) continue;
        const uint64_t own = pe != s->pools.end() ? pool_bytes(pe->second) : 0;
        uint64_t others = resident_bytes(s) - own;
        const uint64_t need = std::max<uint64_t>(q.projected, own);
        if (others + need > s->budget) {
            // evict idle pools, least recently used first, other than this query's
            std::vector<std::pair<double, PoolKey>> idle;
            for (auto& kv : s->pools)
                if (!kv.second.busy && kv.first != key_of(q)) idle.push_back({kv.second.last_used, kv.first});
            std::sort(idle.begin(), idle.end());
            for (auto& c : idle) {
                if (others + need <= s->budget) break;
                auto& e = s->pools[c.second];
                others -= pool_bytes(e);
                hbx_pool_destroy(e.pool);
                s->pools.erase(c.second);
            }
            if (others + need > s->budget) continue;  // wait for running queries
        }
        std::shared_ptr<Query> out = *it;
        s->queue.erase(it);
        return out;
    }
    return nullptr;
}

void worker(hbx_server* s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        std::shared_ptr<Query> q;
        s->cv_work.wait(lock, [&] { return s->stop || (q = pick(s)) != nullptr; });
        if (!q) return;  // stopping
        q->state = Q_RUNNING;
        const PoolKey key = key_of(*q);
        PoolEntry& e = s->pools[key];
        e.busy = true;
        hbx_pool* p = e.pool;
        lock.unlock();

        int rc = HBX_OK;
        if (!p) {
            rc = hbx_pool_create(s->ctx, q->g, q->model, q->seed, &q->o, &p);
            if (rc == HBX_OK) {
                // the pool's first buffers were cleared on the context's stream
                cudaStreamSynchronize(s->ctx->stream);
                cudaStream_t st;
                if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
                    p->stream = st;
                    p->own_stream = true;
                }
            }
        }
        q->seeds.assign(q->k, 0);
        if (rc == HBX_OK)
            rc = imm_on_pool(p, q->k, q->eps, q->ell, q->seeds.data(), &q->influence, nullptr, &q->stats);

        lock.lock();
        PoolEntry& e2 = s->pools[key];
        e2.pool = p;
        e2.busy = false;
        e2.last_used = now_s();
        if (rc == HBX_OK) e2.last_lb = std::max(e2.last_lb, q->stats.lb);
        q->rc = rc;
        if (rc != HBX_OK) {
            std::lock_guard<std::mutex> elock(s->ctx->mu);
            q->error = s->ctx->last_error;
        }
        q->t_done = now_s();
        q->state = Q_DONE;
        s->cv_done.notify_all();
        s->cv_work.notify_all();  // the pool is free again
    }
}

}  // namespace

void hbx_server_destroy_all(hbx_ctx* c) {
    std::vector<hbx_server*> ss;
    {
        std::lock_guard<std::mutex> lock(c->mu);
        ss.assign(c->servers.begin(), c->servers.end());
    }
    for (hbx_server* s : ss) hbx_server_destroy(s);
}

extern "C" int hbx_server_create(hbx_ctx* ctx, uint32_t max_inflight, uint64_t budget, hbx_server** out) {
    if (!ctx || !out || max_inflight == 0 || max_inflight > 64) return HBX_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(ctx, HBX_ERR_CUDA, "cudaMemGetInfo");
        budget = (uint64_t)(0.9 * (double)fr);
    }
    hbx_server* s = new hbx_server();
    s->ctx = ctx;
    s->max_inflight = max_inflight;
    s->budget = budget;
    for (uint32_t i = 0; i < max_inflight; i++) s->workers.emplace_back(worker, s);
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->servers.insert(s);
    }
    *out = s;
    return HBX_OK;
}

extern "C" void hbx_server_destroy(hbx_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (auto& q : s->queue) {
            q->state = Q_CANCELLED;
            q->rc = HBX_ERR_CANCELLED;
        }
        s->queue.clear();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->pools)
        if (kv.second.pool) hbx_pool_destroy(kv.second.pool);
    {
        std::lock_guard<std::mutex> lock(s->ctx->mu);
        s->ctx->servers.erase(s);
    }
    delete s;
}

extern "C" int hbx_submit(hbx_server* s, hbx_graph* g, hbx_model model, uint32_t k, double eps, double ell,
                          uint64_t seed, const hbx_options* opts, hbx_ticket** out) {
    if (!s || !g || !out) return HBX_ERR_INVALID_ARG;
    *out = nullptr;
    auto q = std::make_shared<Query>();
    q->g = g;
    q->model = model;
    q->k = k;
    q->eps = eps;
    q->ell = ell;
    q->seed = seed;
    hbx_default_options(&q->o);
    if (opts) q->o = *opts;
    if (q->o.density_cut == 0) q->o.density_cut = 32;
    double lp, ls;
    if (!imm_lambda(g->n, k, eps, ell, &lp, &ls)) return fail(s->ctx, HBX_ERR_INVALID_ARG, "bad k, eps, ell or n");
    if ((model == HBX_IC && !g->thr) || (model == HBX_LT && !g->q) || (model != HBX_IC && model != HBX_LT))
        return fail(s->ctx, HBX_ERR_INVALID_ARG, "graph lacks the model's parameters");
    if (q->o.encode && q->o.warmup_sets == 0) {
        // fix the warm-up block of a served pool independently of the query:
        // ceil(T_1 / 8) for the reference bounds k = 1, eps = 0.5, ell = 1
        double lp1, ls1;
        imm_lambda(g->n, 1, 0.5, 1.0, &lp1, &ls1);
        const uint64_t T1 = (uint64_t)std::ceil(lp1 / ((double)g->n / 2.0));
        q->o.warmup_sets = (uint32_t)std::min<uint64_t>((T1 + 7) / 8, 0xFFFFFFFFull);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    q->projected = project(s, *q);
    if (q->projected > s->budget)
        return fail(s->ctx, HBX_ERR_ADMISSION,
                    "projected footprint " + std::to_string(q->projected) + " B exceeds the budget");
    q->t_submit = now_s();
    s->queue.push_back(q);
    hbx_ticket* t = new hbx_ticket();
    t->s = s;
    t->q = q;
    *out = t;
    s->cv_work.notify_one();
    return HBX_OK;
}

extern "C" int hbx_wait(hbx_ticket* t, uint32_t* seeds_out, double* influence_out, hbx_stats* stats_out,
                        double* latency_s, int64_t timeout_us) {
    if (!t || !t->q) return HBX_ERR_INVALID_ARG;
    hbx_server* s = t->s;
    std::unique_lock<std::mutex> lock(s->mu);
    auto done = [&] { return t->q->state == Q_DONE || t->q->state == Q_CANCELLED; };
    if (timeout_us < 0) s->cv_done.wait(lock, done);
    else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), done)) return HBX_ERR_TIMEOUT;
    Query& q = *t->q;
    if (q.state == Q_CANCELLED) return HBX_ERR_CANCELLED;
    if (q.rc != HBX_OK) {
        fail(s->ctx, q.rc, q.error);  // the query's own message becomes the context's last error
        return q.rc;
    }
    if (seeds_out) std::copy(q.seeds.begin(), q.seeds.end(), seeds_out);
    if (influence_out) *influence_out = q.influence;
    if (stats_out) *stats_out = q.stats;
    if (latency_s) *latency_s = q.t_done - q.t_submit;
    return HBX_OK;
}

extern "C" int hbx_cancel(hbx_ticket* t) {
    if (!t || !t->q) return HBX_ERR_INVALID_ARG;
    hbx_server* s = t->s;
    std::lock_guard<std::mutex> lock(s->mu);
    if (t->q->state != Q_QUEUED) return HBX_ERR_INVALID_ARG;  // running or finished
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (*it == t->q) {
            s->queue.erase(it);
            break;
        }
    t->q->state = Q_CANCELLED;
    t->q->rc = HBX_ERR_CANCELLED;
    s->cv_done.notify_all();
    return HBX_OK;
}

extern "C" void hbx_ticket_destroy(hbx_ticket* t) { delete t; }
