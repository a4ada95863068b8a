// Serving runtime for resident DtN operators (the solve stage of Section 1.1 under load).
//
// A server owns operators added to it, admits them against a device-memory budget
// (evicting the least recently used ones), and runs two worker threads:
//   - the solve worker, on a high-priority stream, takes every pending solve request
//     whose operator exists when it wakes, groups them by operator and stages each
//     operator's vectors contiguously, then applies ALL of them in one gm_solve_many
//     call -- one launch per precision class over the vectors of every operator in the
//     batch (continuous batching across operators) -- and scatters the results back;
//   - the build worker, on a low-priority stream, runs build requests one at a time while
//     solves go on (the device overlaps the two), then admits each built operator under
//     the budget with the id reserved at submission.  Solves queued for an operator that
//     is still being built wait in the queue until it is admitted (or has failed).
// A request's latency is measured from its submission to the host seeing its result.
// Completion callbacks run on the worker that finished the request, outside the lock;
// gm_server_sync and gm_server_set_callback wait until no callback is running (unless
// called from a callback, which would otherwise wait for itself).
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
    int busy;  // being served by the solve worker: never evicted meanwhile
};

}  // namespace

struct gm_server {
    int device = 0;
    long long budget = 0, used = 0;
    int batching = 1;
    cudaStream_t stream = nullptr;   // solves (highest priority)
    cudaStream_t bstream = nullptr;  // builds (lowest priority)
    std::mutex mu;
    std::condition_variable cv_work, cv_build, cv_done;
    std::deque<Request> queue;   // solve requests
    std::deque<Request> bqueue;  // build requests
    std::map<int, Operator> ops;
    std::set<int> building;  // ids reserved by build requests not yet finished
    gm_server_callback cb = nullptr;  // called for every completed request (worker threads)
    void *cb_user = nullptr;
    int cb_running = 0;  // callbacks in progress
    std::map<long long, int> status;  // request id -> result code once completed
    int next_op = 1;
    long long next_req = 1, tick = 0;
    bool stop = false;
    int in_flight = 0, b_in_flight = 0;
    // statistics
    std::vector<double> lat_ms;
    long long vectors = 0, solves = 0, evictions = 0;
    Clock::time_point first_submit{}, last_done{};
    bool any = false;
    std::thread worker, builder;
    std::thread::id worker_id, builder_id;
    // device staging of the batched solve (grown on demand, solve-worker-owned)
    double *dg = nullptr, *dv = nullptr;
    size_t cap = 0;

    bool on_worker() const {
        const std::thread::id me = std::this_thread::get_id();
        return me == worker_id || me == builder_id;
    }

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

    // A build request: the operator is built on the build stream, then admitted under the
    // budget with the id reserved at submission.  Called with mu held; unlocks it during
    // the build.
    int run_build(const Request &r, std::unique_lock<std::mutex> &lk) {
        gm_opts o = r.opts;
        o.stream = bstream;
        o.background = 1;
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

    // Every operator's requests of one batch: one grouped solve over all of them (each
    // operator's vectors concatenated), or, unbatched, one solve per request.  rc[i] is
    // operator i's result.
    void serve(const std::vector<Operator> &opv, const std::vector<std::vector<Request>> &rq, std::vector<int> &rc) {
        const size_t no = opv.size();
        rc.assign(no, GM_OK);
        if (!batching) {  // the unbatched baseline: one solve per request
            for (size_t i = 0; i < no; ++i)
                for (const Request &r : rq[i])
                    if (rc[i] == GM_OK) rc[i] = gm_solve(opv[i].h, r.g, r.dudn, r.batch, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess)
                for (int &x : rc)
                    if (x == GM_OK) x = GM_ECUDA;
            return;
        }
        std::vector<size_t> at(no + 1, 0);
        std::vector<int> tot(no, 0);
        for (size_t i = 0; i < no; ++i) {
            for (const Request &r : rq[i]) tot[i] += r.batch;
            at[i + 1] = at[i] + 4 * (size_t)opv[i].n * tot[i];
        }
        int e = ensure(at[no]);
        std::vector<gm_handle *> hs(no);
        std::vector<const double *> gp(no);
        std::vector<double *> vp(no);
        for (size_t i = 0; i < no && e == GM_OK; ++i) {
            const size_t N = 4 * (size_t)opv[i].n;
            size_t off = at[i];
            for (const Request &r : rq[i]) {
                if (cudaMemcpyAsync(dg + off, r.g, N * r.batch * 8, cudaMemcpyDefault, stream) != cudaSuccess)
                    e = GM_ECUDA;
                off += N * r.batch;
            }
            hs[i] = opv[i].h;
            gp[i] = dg + at[i];
            vp[i] = dv + at[i];
        }
        if (e == GM_OK) {
            e = gm_solve_many((int)no, hs.data(), gp.data(), vp.data(), tot.data(), stream);
            if (e != GM_OK && no > 1)  // find which operators fail: each alone
                for (size_t i = 0; i < no; ++i) rc[i] = gm_solve_many(1, &hs[i], &gp[i], &vp[i], &tot[i], stream);
            else
                rc.assign(no, e);
        } else {
            rc.assign(no, e);
        }
        for (size_t i = 0; i < no; ++i) {
            if (rc[i] != GM_OK) continue;
            const size_t N = 4 * (size_t)opv[i].n;
            size_t off = at[i];
            for (const Request &r : rq[i]) {
                if (cudaMemcpyAsync(r.dudn, dv + off, N * r.batch * 8, cudaMemcpyDefault, stream) != cudaSuccess)
                    rc[i] = GM_ECUDA;
                off += N * r.batch;
            }
        }
        if (cudaStreamSynchronize(stream) != cudaSuccess)
            for (int &x : rc)
                if (x == GM_OK) x = GM_ECUDA;
    }

    // Callbacks for completed requests, outside the lock; mu held on entry and exit.
    void notify(std::unique_lock<std::mutex> &lk, const std::vector<long long> &ids) {
        const gm_server_callback call = cb;
        void *const user = cb_user;
        if (call) ++cb_running;
        cv_done.notify_all();
        if (!call) return;
        std::vector<std::pair<long long, int>> done;
        for (long long id : ids) done.push_back({id, status[id]});
        lk.unlock();
        for (const auto &q : done) call(q.first, q.second, user);
        lk.lock();
        --cb_running;
        cv_done.notify_all();
    }

    bool ready(const Request &r) const { return !building.count(r.op); }

    void run_solves() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_work.wait(lk, [&] {
                if (stop) return true;
                for (const Request &r : queue)
                    if (ready(r)) return true;
                return false;
            });
            std::vector<Request> take;
            std::deque<Request> keep;
            for (const Request &r : queue) (ready(r) ? take.push_back(r) : keep.push_back(r));
            if (take.empty() && stop) break;
            queue.swap(keep);
            in_flight = (int)take.size();
            // group by operator, in order of first arrival
            std::vector<int> order;
            std::map<int, std::vector<Request>> by_op;
            for (const Request &r : take) {
                if (!by_op.count(r.op)) order.push_back(r.op);
                by_op[r.op].push_back(r);
            }
            std::vector<Operator> opv;
            std::vector<std::vector<Request>> rq;
            std::vector<int> ids;
            for (int id : order) {
                auto it = ops.find(id);
                if (it == ops.end()) {  // evicted after the request was queued, or its build failed
                    for (const Request &r : by_op[id]) status[r.id] = GM_EINVAL;
                    continue;
                }
                it->second.last_use = ++tick;
                it->second.busy = 1;
                opv.push_back(it->second);
                rq.push_back(by_op[id]);
                ids.push_back(id);
            }
            std::vector<int> rc;
            if (!opv.empty()) {
                lk.unlock();
                serve(opv, rq, rc);
                lk.lock();
                ++solves;
            }
            const Clock::time_point done = Clock::now();
            for (size_t i = 0; i < ids.size(); ++i) {
                ops[ids[i]].busy = 0;
                for (const Request &r : rq[i]) {
                    status[r.id] = rc[i];
                    if (rc[i] == GM_OK) {
                        lat_ms.push_back(std::chrono::duration<double, std::milli>(done - r.t_submit).count());
                        vectors += r.batch;
                        last_done = done;
                    }
                }
            }
            in_flight = 0;
            std::vector<long long> fin;
            for (const Request &r : take) fin.push_back(r.id);
            notify(lk, fin);
        }
    }

    void run_builds() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            cv_build.wait(lk, [&] { return stop || !bqueue.empty(); });
            if (stop) break;
            const Request r = bqueue.front();
            bqueue.pop_front();
            b_in_flight = 1;
            const int rc = run_build(r, lk);
            status[r.id] = rc;
            building.erase(r.op);
            last_done = Clock::now();
            b_in_flight = 0;
            cv_work.notify_all();  // solves queued for this operator may run now
            notify(lk, {r.id});
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
    int lo = 0, hi = 0;  // numerically lower = higher priority
    if (cudaGetDevice(&s->device) != cudaSuccess || cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->bstream, cudaStreamNonBlocking, lo) != cudaSuccess) {
        cudaGetLastError();
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return GM_ECUDA;
    }
    s->worker = std::thread([s] { s->run_solves(); });
    s->builder = std::thread([s] { s->run_builds(); });
    s->worker_id = s->worker.get_id();
    s->builder_id = s->builder.get_id();
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
    if (!s || !b || !c || !d || n < 2 || leaf < 3 || !(tol >= 0.0) || !op_id || !req_id) return GM_EINVAL;
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
    s->bqueue.push_back(r);
    *op_id = r.op;
    *req_id = r.id;
    s->cv_build.notify_one();
    return GM_OK;
}

int gm_server_set_callback(gm_server *s, gm_server_callback cb, void *user) {
    if (!s) return GM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cb = cb;
    s->cb_user = user;
    // a callback already started with the previous function finishes before this returns
    if (!s->on_worker()) s->cv_done.wait(lk, [&] { return s->cb_running == 0; });
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
    const bool mine = s->on_worker();
    s->cv_done.wait(lk, [&] {
        return s->queue.empty() && s->bqueue.empty() && s->in_flight == 0 && s->b_in_flight == 0 &&
               (mine || s->cb_running == 0);
    });
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
        s->cv_build.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->builder.joinable()) s->builder.join();
    for (auto &kv : s->ops) gm_free(kv.second.h);
    if (s->dg) cudaFree(s->dg);
    if (s->dv) cudaFree(s->dv);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->bstream) cudaStreamDestroy(s->bstream);
    delete s;
}

}  // extern "C"
