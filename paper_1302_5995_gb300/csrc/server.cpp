// Serving runtime for resident DtN operators (the solve stage of Section 1.1 under load).
//
// A server owns operators added to it, admits them against a device-memory budget
// (evicting the least recently used ones), and runs one worker thread with its own
// stream.  Clients submit solve requests (any number of vectors for one operator) and
// return immediately; the worker takes every request pending when it wakes, groups them
// by operator and runs ONE solve per operator over the concatenated vectors (continuous
// batching), then scatters the results back.  A request's latency is measured from its
// submission to the host seeing its result complete.  Build requests run on the worker
// too, before the solves taken with them, and admit their operator under the budget
// with the id reserved at submission (solves may be queued for it at once).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "../../include/gm.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id;
    int op;
    const double *g;
    double *dudn;
    int batch;
    Clock::time_point t_submit;
    // a build request (op is the id reserved for the new operator)
    bool build = false;
    gm_opts opts{};
    const double *b = nullptr, *c = nullptr, *d = nullptr;
    int n = 0, leaf = 0;
    double tol = 0.0;
};

struct Operator {
    gm_handle *h;
    int n;
    long long bytes;
    long long last_use;
    int busy;  // being served by the worker: never evicted meanwhile
};

}  // namespace

struct gm_server {
    int device = 0;
    long long budget = 0, used = 0;
    int batching = 1;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::map<int, Operator> ops;
    std::set<int> building;  // ids reserved by build requests not yet finished
    gm_server_callback cb = nullptr;  // called for every completed request (worker thread)
    void *cb_user = nullptr;
    std::map<long long, int> status;  // request id -> result code once completed
    int next_op = 1;
    long long next_req = 1, tick = 0;
    bool stop = false;
    int in_flight = 0;
    // statistics
    std::vector<double> lat_ms;
    long long vectors = 0, solves = 0, evictions = 0;
    Clock::time_point first_submit{}, last_done{};
    bool any = false;
    std::thread worker;
    // device staging of the batched solve (grown on demand, worker-owned)
    double *dg = nullptr, *dv = nullptr;
    size_t cap = 0;

    int ensure(size_t doubles) {
        if (doubles <= cap) return GM_OK;
        if (dg) cudaFree(dg);
        if (dv) cudaFree(dv);
        dg = dv = nullptr;
        cap = 0;
        if (cudaMalloc(&dg, doubles * 8) != cudaSuccess || cudaMalloc(&dv, doubles * 8) != cudaSuccess) {
            cudaGetLastError();
            return GM_ENOMEM;
        }
        cap = doubles;
        return GM_OK;
    }

    // Evict least recently used operators (never one being served) until `need` more
    // bytes fit the budget; false if that is impossible.  Called with mu held.
    bool room_for(long long need) {
        while (used + need > budget) {
            auto victim = ops.end();
            for (auto it = ops.begin(); it != ops.end(); ++it)
                if (!it->second.busy && (victim == ops.end() || it->second.last_use < victim->second.last_use))
                    victim = it;
            if (victim == ops.end()) return false;
            used -= victim->second.bytes;
            gm_free(victim->second.h);
            ops.erase(victim);
            ++evictions;
        }
        return true;
    }

    // A build request: the operator is built on the worker's stream, then admitted under
    // the budget with the id reserved at submission.  Called with mu held; unlocks it
    // during the build.
    int run_build(const Request &r, std::unique_lock<std::mutex> &lk) {
        gm_opts o = r.opts;
        o.stream = stream;
        gm_handle *h = nullptr;
        lk.unlock();
        int rc = gm_build_ex(&o, r.b, r.c, r.d, r.n, r.leaf, r.tol, &h);
        gm_info_t inf;
        if (rc == GM_OK && (rc = gm_info(h, &inf)) != GM_OK) gm_free(h);
        lk.lock();
        if (rc != GM_OK) return rc;
        const long long bytes = inf.resident_bytes;
        if (bytes > budget || !room_for(bytes)) {
            gm_free(h);
            return GM_ENOMEM;
        }
        ops[r.op] = Operator{h, inf.n, bytes, ++tick, 0};
        used += bytes;
        return GM_OK;
    }

    // Run one operator's requests as one solve over their concatenated vectors.
    int serve(const Operator &op, const std::vector<Request> &rq) {
        const size_t N = 4 * (size_t)op.n;
        if (!batching) {  // the unbatched baseline: one solve per request
            for (const Request &r : rq) {
                const int rc = gm_solve(op.h, r.g, r.dudn, r.batch, stream);
                if (rc) return rc;
            }
            return cudaStreamSynchronize(stream) == cudaSuccess ? GM_OK : GM_ECUDA;
        }
        size_t total = 0;
        for (const Request &r : rq) total += (size_t)r.batch;
        int rc = ensure(N * total);
        if (rc) return rc;
        size_t at = 0;
        for (const Request &r : rq) {
            if (cudaMemcpyAsync(dg + at * N, r.g, N * r.batch * 8, cudaMemcpyDefault, stream) != cudaSuccess)
                return GM_ECUDA;
            at += r.batch;
        }
        if ((rc = gm_solve(op.h, dg, dv, (int)total, stream))) return rc;
        at = 0;
        for (const Request &r : rq) {
            if (cudaMemcpyAsync(r.dudn, dv + at * N, N * r.batch * 8, cudaMemcpyDefault, stream) != cudaSuccess)
                return GM_ECUDA;
            at += r.batch;
        }
        return cudaStreamSynchronize(stream) == cudaSuccess ? GM_OK : GM_ECUDA;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            if (queue.empty() && stop) break;
            std::vector<Request> take(queue.begin(), queue.end());
            queue.clear();
            in_flight = (int)take.size();
            const gm_server_callback call = cb;
            void *const user = cb_user;
            // builds first, in arrival order, so that solves queued behind a build find it
            for (const Request &r : take)
                if (r.build) {
                    status[r.id] = run_build(r, lk);
                    building.erase(r.op);
                    last_done = Clock::now();
                }
            // solves grouped by operator, in order of first arrival
            std::vector<int> order;
            std::map<int, std::vector<Request>> by_op;
            for (const Request &r : take) {
                if (r.build) continue;
                if (!by_op.count(r.op)) order.push_back(r.op);
                by_op[r.op].push_back(r);
            }
            for (int id : order) {
                auto it = ops.find(id);
                std::vector<Request> &rq = by_op[id];
                int rc = GM_EINVAL;  // the operator was evicted after the request was queued
                if (it != ops.end()) {
                    it->second.last_use = ++tick;
                    it->second.busy = 1;
                    const Operator op = it->second;
                    lk.unlock();
                    rc = serve(op, rq);
                    lk.lock();
                    ops[id].busy = 0;
                    ++solves;
                }
                const Clock::time_point done = Clock::now();
                for (const Request &r : rq) {
                    status[r.id] = rc;
                    if (rc == GM_OK) {
                        lat_ms.push_back(std::chrono::duration<double, std::milli>(done - r.t_submit).count());
                        vectors += r.batch;
                        last_done = done;
                    }
                }
            }
            in_flight = 0;
            cv_done.notify_all();
            if (call) {  // outside the lock: the callback may call back into the server
                std::vector<std::pair<long long, int>> done;
                for (const Request &r : take) done.push_back({r.id, status[r.id]});
                lk.unlock();
                for (const auto &q : done) call(q.first, q.second, user);
                lk.lock();
            }
        }
    }
};

namespace {

bool make_room(gm_server *s, long long need) { return s->room_for(need); }

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int gm_server_create(long long budget_bytes, int batching, gm_server **out) {
    if (!out || budget_bytes <= 0) return GM_EINVAL;
    *out = nullptr;
    gm_server *s = new gm_server();
    s->budget = budget_bytes;
    s->batching = batching ? 1 : 0;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return GM_ECUDA;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return GM_OK;
}

int gm_server_add(gm_server *s, gm_handle *h, int *op_id) {
    if (!s || !h || !op_id) return GM_EINVAL;
    gm_info_t inf;
    int rc = gm_info(h, &inf);
    if (rc) return rc;
    const long long bytes = inf.resident_bytes;
    std::lock_guard<std::mutex> lk(s->mu);
    if (bytes > s->budget || !make_room(s, bytes)) return GM_ENOMEM;
    const int id = s->next_op++;
    s->ops[id] = Operator{h, inf.n, bytes, ++s->tick, 0};
    s->used += bytes;
    *op_id = id;
    return GM_OK;
}

int gm_server_submit(gm_server *s, int op_id, const double *g, double *dudn, int batch, long long *req_id) {
    if (!s || !g || !dudn || batch <= 0 || !req_id) return GM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->ops.count(op_id) && !s->building.count(op_id)) return GM_EINVAL;
    Request r{s->next_req++, op_id, g, dudn, batch, Clock::now()};
    if (!s->any) {
        s->first_submit = r.t_submit;
        s->any = true;
    }
    s->queue.push_back(r);
    *req_id = r.id;
    s->cv_work.notify_one();
    return GM_OK;
}

int gm_server_submit_build(gm_server *s, const gm_opts *opts, const double *b, const double *c, const double *d,
                           int n, int leaf, double tol, int *op_id, long long *req_id) {
    if (!s || !b || !c || !d || n < 2 || leaf < 4 || !(tol >= 0.0) || !op_id || !req_id) return GM_EINVAL;
    Request r{0, 0, nullptr, nullptr, 0, Clock::now()};
    r.build = true;
    gm_opts_default(&r.opts);
    if (opts) r.opts = *opts;
    r.b = b;
    r.c = c;
    r.d = d;
    r.n = n;
    r.leaf = leaf;
    r.tol = tol;
    std::lock_guard<std::mutex> lk(s->mu);
    r.id = s->next_req++;
    r.op = s->next_op++;
    s->building.insert(r.op);
    s->queue.push_back(r);
    *op_id = r.op;
    *req_id = r.id;
    s->cv_work.notify_one();
    return GM_OK;
}

int gm_server_set_callback(gm_server *s, gm_server_callback cb, void *user) {
    if (!s) return GM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->cb = cb;
    s->cb_user = user;
    return GM_OK;
}

int gm_server_poll(gm_server *s, long long req_id, int *done) {
    if (!s || !done) return GM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (req_id <= 0 || req_id >= s->next_req) return GM_EINVAL;
    auto it = s->status.find(req_id);
    *done = it != s->status.end();
    return *done ? it->second : GM_OK;
}

int gm_server_wait(gm_server *s, long long req_id) {
    if (!s) return GM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (req_id <= 0 || req_id >= s->next_req) return GM_EINVAL;
    s->cv_done.wait(lk, [&] { return s->status.count(req_id) > 0; });
    return s->status[req_id];
}

int gm_server_sync(gm_server *s) {
    if (!s) return GM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->queue.empty() && s->in_flight == 0; });
    return GM_OK;
}

int gm_server_stats(gm_server *s, gm_server_stats_t *st) {
    if (!s || !st) return GM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->requests = (long long)s->lat_ms.size();
    st->vectors = s->vectors;
    st->solves = s->solves;
    st->evictions = s->evictions;
    st->resident_ops = (int)s->ops.size();
    st->resident_bytes = s->used;
    st->p50_ms = percentile(s->lat_ms, 0.50);
    st->p99_ms = percentile(s->lat_ms, 0.99);
    const double span = s->any ? std::chrono::duration<double>(s->last_done - s->first_submit).count() : 0.0;
    st->vectors_per_s = span > 0.0 ? (double)s->vectors / span : 0.0;
    return GM_OK;
}

int gm_server_reset_stats(gm_server *s) {
    if (!s) return GM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->vectors = s->solves = s->evictions = 0;
    s->any = false;
    return GM_OK;
}

void gm_server_destroy(gm_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->ops) gm_free(kv.second.h);
    if (s->dg) cudaFree(s->dg);
    if (s->dv) cudaFree(s->dv);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
