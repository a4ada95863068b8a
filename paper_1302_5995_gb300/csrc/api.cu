// C ABI: gm_build / gm_build_batch / gm_solve / gm_get_dtn / gm_get_schur / gm_info / gm_free.
//
// A build runs the paper's level-by-level sweep (Section 3.3): every leaf of every
// problem in one launch, then per tree level one stage of horizontal pairwise merges and
// one of vertical ones -- each stage one batch over all its merges, across all problems
// of a batched build (stages aligned from the root) -- then all roots in one batch.
// Every Schur complement of a build lives in one device arena; the rest of the device
// memory comes from the stream-ordered allocator on the build stream.
#include <cuda_runtime.h>

#include <chrono>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "blocked.h"
#include "gm_internal.h"
#include "hbs.h"
#include "kernels.h"
#include "loads.h"
#include "mixed.h"
#include "network.h"

using namespace gm;

namespace {

// With GM_DEBUG set in the environment, every failing CUDA call is reported on stderr
// with its source line and the runtime's error string.
bool debug_on() {
    static const bool on = getenv("GM_DEBUG") != nullptr;
    return on;
}

// Runs job(j, stream) for j in [0, count) on up to kMaxLanes host threads, each with a
// stream of its own (created once per device) that first waits for what `s` has queued;
// `s` then waits for all of them.  For independent, host-synchronising work (the HBS
// factorisations of the merges of a stage).  Returns GM_ECUDA if the streams or events
// could not be set up; the jobs report their own results.
constexpr int kMaxLanes = 16;
template <class Job>
int run_lanes(int count, cudaStream_t s, Job job) {
    struct Lanes {
        cudaStream_t st[kMaxLanes] = {};
        cudaEvent_t done[kMaxLanes] = {};
        cudaEvent_t start = nullptr;
        bool ok = false;
    };
    static std::mutex mu;
    static std::map<int, Lanes> by_dev;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GM_ECUDA;
    }
    Lanes *L;
    {
        std::lock_guard<std::mutex> lk(mu);
        L = &by_dev[dev];
        if (!L->ok) {
            bool good = cudaEventCreateWithFlags(&L->start, cudaEventDisableTiming) == cudaSuccess;
            for (int i = 0; good && i < kMaxLanes; ++i)
                good = cudaStreamCreateWithFlags(&L->st[i], cudaStreamNonBlocking) == cudaSuccess &&
                       cudaEventCreateWithFlags(&L->done[i], cudaEventDisableTiming) == cudaSuccess;
            if (!good) {
                cudaGetLastError();
                return GM_ECUDA;
            }
            L->ok = true;
        }
    }
    // one build at a time uses the lanes of a device
    static std::mutex use_mu;
    std::lock_guard<std::mutex> use(use_mu);
    const int nl = std::min(count, kMaxLanes);
    if (cudaEventRecord(L->start, s) != cudaSuccess) return GM_ECUDA;
    for (int i = 0; i < nl; ++i)
        if (cudaStreamWaitEvent(L->st[i], L->start, 0) != cudaSuccess) return GM_ECUDA;
    std::atomic<int> next(0);
    std::vector<std::thread> th;
    for (int i = 0; i < nl; ++i)
        th.emplace_back([&, i] {
            cudaSetDevice(dev);
            for (int j = next++; j < count; j = next++) job(j, L->st[i]);
            cudaEventRecord(L->done[i], L->st[i]);
        });
    for (auto &t : th) t.join();
    for (int i = 0; i < nl; ++i)
        if (cudaStreamWaitEvent(s, L->done[i], 0) != cudaSuccess) return GM_ECUDA;
    return GM_OK;
}

// GM_TUNE (environment, read at every build) forces launch shapes and schedules, so that
// every variant the autotuner may choose can be tested: comma-separated key=value pairs
// of rtile32_max, tc_min_k, early, a11, upd_tiles (e.g. "early=1,upd_tiles=-1").
void tune_override(Tune &t) {
    const char *env = getenv("GM_TUNE");
    if (!env || !*env) return;
    std::string s(env);
    size_t at = 0;
    while (at < s.size()) {
        size_t end = s.find(',', at);
        if (end == std::string::npos) end = s.size();
        const std::string kv = s.substr(at, end - at);
        const size_t eq = kv.find('=');
        if (eq != std::string::npos) {
            const std::string key = kv.substr(0, eq);
            const int v = atoi(kv.c_str() + eq + 1);
            if (key == "rtile32_max") t.rtile32_max = v;
            else if (key == "tc_min_k") t.tc_min_k = v;
            else if (key == "early") t.early = v;
            else if (key == "a11") t.a11 = v;
            else if (key == "upd_tiles") t.upd_tiles = v;
        }
        at = end + 1;
    }
}

// Multiprocessors of the current device (looked up once per device).
int device_sms() {
    static std::mutex mu;
    static std::map<int, int> by_dev;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    std::lock_guard<std::mutex> lk(mu);
    auto it = by_dev.find(dev);
    if (it != by_dev.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 152;
    }
    by_dev[dev] = n;
    return n;
}

int cuda_fail(cudaError_t e, const char *what, int line) {
    if (debug_on()) fprintf(stderr, "gm: api.cu:%d: %s: %s\n", line, what, cudaGetErrorString(e));
    return GM_ECUDA;
}

#define CK(x)                                                  \
    do {                                                       \
        cudaError_t _e = (x);                                  \
        if (_e != cudaSuccess) return cuda_fail(_e, #x, __LINE__); \
    } while (0)

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The library's stream-ordered memory pool on a device: it keeps freed workspace mapped
// (release threshold unbounded), so a build does not map its few hundred MB of temporaries
// anew after every synchronisation, as the device's default pool (threshold 0) would.
// Result code of a failed allocation: GM_ENOMEM when the device is out of memory,
// GM_ECUDA for any other runtime failure (no device, no driver, a sticky error).
int alloc_error(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GM_ENOMEM : GM_ECUDA;
}

// Allocation-failure injection (gm_debug_fail_alloc): when the countdown reaches 1, that
// device allocation fails as if the device were out of memory.
std::atomic<long long> g_fail_countdown{0};
bool injected_failure() {
    long long c = g_fail_countdown.load();
    while (c > 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

// Allocation context of a build that is recorded into a CUDA graph: while `measure` is
// set, allocations are made as usual and their (aligned) sizes summed; while `base` is set,
// they are carved in order from one buffer that the graph keeps (frees do nothing), so a
// replay finds every buffer where the recording put it.
struct BumpCtx {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    bool measure = false;
    size_t total = 0;
    static size_t align(size_t b) { return (b + 255) / 256 * 256; }
    bool bumping() const { return base != nullptr; }
    void *take(size_t bytes) {
        const size_t a = align(bytes);
        if (used + a > cap) return nullptr;
        void *p = base + used;
        used += a;
        return p;
    }
};
thread_local BumpCtx *tl_bump = nullptr;
// the status array of the build being recorded (its replays report through it)
thread_local gm::Status *tl_recorded_status = nullptr;

// cudaMalloc with the injection point (the handle's long-lived buffers).
cudaError_t lib_malloc(void **p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    if (tl_bump && tl_bump->bumping()) {
        *p = tl_bump->take(bytes);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    if (tl_bump && tl_bump->measure) tl_bump->total += BumpCtx::align(bytes);
    return cudaMalloc(p, bytes);
}

cudaMemPool_t lib_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = pool;
    return pool;
}

// Device buffer released on scope exit through the stream-ordered allocator (or carved
// from a graph's buffer while a build is being recorded: see BumpCtx).
struct DBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    bool bumped = false;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p && !bumped) cudaFreeAsync(p, s);
        p = nullptr;
        bumped = false;
    }
    int alloc(size_t bytes, cudaStream_t st) {
        release();
        s = st;
        if (bytes == 0) bytes = 16;
        if (injected_failure()) return GM_ENOMEM;
        if (tl_bump && tl_bump->bumping()) {
            p = tl_bump->take(bytes);
            bumped = p != nullptr;
            return p ? GM_OK : GM_ENOMEM;
        }
        if (tl_bump && tl_bump->measure) tl_bump->total += BumpCtx::align(bytes);
        cudaMemPool_t pool = lib_pool();
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            p = nullptr;
            return alloc_error(e);
        }
        return GM_OK;
    }
    template <class T> T *as() const { return (T *)p; }
};

// Streams and events for the look-ahead of the blocked sweep (released on scope exit,
// after the build has synchronised): s1 carries the critical chain at the highest
// priority, s2 the bulk of each update at the lowest.
struct LookAhead {
    cudaStream_t s1 = nullptr, s2 = nullptr, s3 = nullptr;
    cudaEvent_t a = nullptr, b = nullptr, c = nullptr, d = nullptr, e = nullptr, f[2] = {nullptr, nullptr};
    ~LookAhead() {
        if (s1) cudaStreamSynchronize(s1);
        if (s2) cudaStreamSynchronize(s2);
        if (s3) cudaStreamSynchronize(s3);
        for (cudaEvent_t x : {a, b, c, d, e, f[0], f[1]})
            if (x) cudaEventDestroy(x);
        if (s1) cudaStreamDestroy(s1);
        if (s2) cudaStreamDestroy(s2);
        if (s3) cudaStreamDestroy(s3);
    }
    // background: both streams at the lowest priority (the build yields to other work)
    bool create(bool background) {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s1, cudaStreamNonBlocking, background ? least : greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s3, cudaStreamNonBlocking, background ? least : greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&d, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&f[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&f[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }
};

// Device copy of a plan (cached per device and per list of (n, leaf)).
struct DevStage {
    int orient, nm, max_m, max_ncol, max_rp;
    int sum_rows = 0, sum_cols = 0;
    int64_t out_base, out_doubles, ws_doubles, max_elems, dig_elems, exp_elems;
    MergeDesc *d_merges = nullptr;
    int *d_tab = nullptr;
    SysDesc *d_sys = nullptr;
    std::vector<SysDesc> h_sys;
};
struct DevPlan {
    Plan plan;
    LeafDesc *d_leaves = nullptr;
    int max_leaf_a = 0, max_leaf_b = 0;
    std::vector<DevStage> stages;
    SysDesc *d_root_sys = nullptr;
    std::vector<SysDesc> h_root_sys;
    int64_t root_ws = 0;  // elements of the roots' dense systems
    int max_root_ncol = 0;
    ~DevPlan() {
        cudaFree(d_leaves);
        for (auto &s : stages) {
            cudaFree(s.d_merges);
            cudaFree(s.d_tab);
            cudaFree(s.d_sys);
        }
        cudaFree(d_root_sys);
    }
};

using PlanKey = std::pair<int, std::vector<std::pair<int, int>>>;
std::mutex g_plan_mu;
std::map<PlanKey, std::shared_ptr<DevPlan>> g_plans;

template <class T> int upload(T **dst, const std::vector<T> &v) {
    size_t bytes = v.size() * sizeof(T);
    const cudaError_t e = lib_malloc((void **)dst, bytes ? bytes : 16);
    if (e != cudaSuccess) return alloc_error(e);
    if (bytes && cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return GM_ECUDA;
    return GM_OK;
}

int make_devplan(DevPlan &dp) {
    int rc;
    const Plan &P = dp.plan;
    for (const LeafDesc &l : P.leaves) {
        dp.max_leaf_a = std::max(dp.max_leaf_a, l.a);
        dp.max_leaf_b = std::max(dp.max_leaf_b, l.b);
    }
    if ((rc = upload(&dp.d_leaves, P.leaves))) return rc;
    for (const Stage &st : P.stages) {
        DevStage ds;
        ds.orient = st.orient;
        ds.nm = (int)st.merges.size();
        ds.max_m = st.max_m;
        ds.max_ncol = st.max_ncol;
        ds.max_rp = st.max_rp;
        ds.out_base = st.out_base;
        ds.out_doubles = st.out_doubles;
        ds.ws_doubles = st.ws_doubles;
        ds.dig_elems = st.dig_elems;
        ds.exp_elems = st.exp_elems;
        ds.max_elems = 0;
        int roff = 0, coff = 0;
        for (int i = 0; i < ds.nm; ++i) {
            const MergeDesc &m = st.merges[i];
            SysDesc s{m.ws, 2 * m.sp, 2 * m.sp + m.rp, i, roff, coff, m.prob};
            roff += s.m;
            coff += s.ncol;
            ds.h_sys.push_back(s);
            ds.max_elems = std::max(ds.max_elems, (int64_t)s.m * s.ncol);
        }
        ds.sum_rows = roff;
        ds.sum_cols = coff;
        dp.stages.push_back(ds);
        DevStage &d = dp.stages.back();
        if ((rc = upload(&d.d_merges, st.merges))) return rc;
        if ((rc = upload(&d.d_tab, st.table))) return rc;
        if ((rc = upload(&d.d_sys, d.h_sys))) return rc;
    }
    int roff = 0, coff = 0;
    int64_t wo = 0;
    for (size_t i = 0; i < P.roots.size(); ++i) {
        const RootDesc &r = P.roots[i];
        SysDesc s{wo, r.r, r.r + 4 * r.n, (int)i, roff, coff, r.problem};
        roff += s.m;
        coff += s.ncol;
        wo += (int64_t)s.m * s.ncol;
        dp.max_root_ncol = std::max(dp.max_root_ncol, s.ncol);
        dp.h_root_sys.push_back(s);
    }
    dp.root_ws = wo;
    return upload(&dp.d_root_sys, dp.h_root_sys);
}

int get_plan(const std::vector<std::pair<int, int>> &probs, std::shared_ptr<DevPlan> &out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    PlanKey key(dev, probs);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        out = it->second;
        return GM_OK;
    }
    auto dp = std::make_shared<DevPlan>();
    int rc;
    if (probs.size() == 1) {
        rc = build_plan(probs[0].first, probs[0].second, dp->plan);
    } else {
        std::vector<Plan> singles(probs.size());
        std::vector<const Plan *> ptrs;
        std::vector<int64_t> coef;
        int64_t acc = 0;
        for (size_t i = 0; i < probs.size(); ++i) {
            if ((rc = build_plan(probs[i].first, probs[i].second, singles[i]))) return rc;
            ptrs.push_back(&singles[i]);
            coef.push_back(acc);
            acc += (int64_t)probs[i].first * probs[i].first;
        }
        rc = build_batch_plan(ptrs, coef, dp->plan);
    }
    if (rc) return rc;
    if ((rc = make_devplan(*dp))) return rc;
    g_plans[key] = dp;
    out = dp;
    return GM_OK;
}

}  // namespace

namespace gm {
static std::mutex g_ev_mu;
static std::vector<cudaEvent_t> g_ev_pool;
cudaEvent_t event_pool_get() {
    {
        std::lock_guard<std::mutex> lk(g_ev_mu);
        if (!g_ev_pool.empty()) {
            cudaEvent_t e = g_ev_pool.back();
            g_ev_pool.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
void event_pool_put(cudaEvent_t e) {
    if (!e) return;
    std::lock_guard<std::mutex> lk(g_ev_mu);
    g_ev_pool.push_back(e);
}
int dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (injected_failure()) return GM_ENOMEM;
    cudaMemPool_t pool = lib_pool();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return alloc_error(e);
    }
    return GM_OK;
}
}  // namespace gm

namespace {
// Status of every problem of a build reset on the device (a recorded build resets it
// itself at every replay).
__global__ void k_status_init(Status *st, int np) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np) st[p] = Status{0, -1, 0x7ff0000000000000ull, 0, 0u};
}

// An open stream capture, ended (and its graph dropped) if the build returns early.
struct CaptureGuard {
    cudaStream_t s = nullptr;
    bool active = false;
    ~CaptureGuard() {
        if (!active) return;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
};
}  // namespace

struct gm_handle {
    int n = 0, leaf = 0, L = 0, precision = 0;
    double *T = nullptr;            // 4n x 4n column-major
    float2 *Tdf = nullptr;          // mixed precision: T as double-float
    __nv_bfloat16 *tdig = nullptr;  // mixed precision: digit planes of T's rows, for the apply
    int *tex = nullptr;             // mixed precision: row exponents of T
    int split = 6;                  // mixed precision: digits per operand
    std::shared_ptr<DevPlan> plan;
    // kept intermediates: box -> device pointer of its Schur complement (FP64, or
    // double-float pairs for a mixed-precision build)
    std::vector<std::pair<Box, void *>> kept;
    bool kept_df32 = false;
    std::vector<void *> kept_bufs;
    gm::HbsRoot *hbs = nullptr;     // tol > 0: the root's HBS inverse (no dense T)
    double *F = nullptr;            // body loads: the 4n x nbody load operator (Section 6.3)
    int nbody = 0;
    double *FL = nullptr, *FR = nullptr;  // F ~ FL FR after gm_compress_load_operator
    int frank = -1;                       // its rank (-1: F is dense)
    gm_info_t info{};
};

const double *gm::handle_dtn(gm_handle *h, int *n) {
    if (!h) return nullptr;
    *n = h->n;
    return h->T;
}

bool gm::handle_split(gm_handle *h, const void **tdig, const int **tex, int *split) {
    if (!h || h->precision != GM_PREC_MIXED || h->hbs || !h->tdig) return false;
    *tdig = h->tdig;
    *tex = h->tex;
    *split = h->split;
    return true;
}

extern "C" void gm_free(gm_handle *h);

namespace {

// Largest refinement ratio of a block solve accepted by the automatic mode (its square,
// about the relative error left by one refinement step, is 2^-26 = 1.5e-8).
constexpr float kMaxRefineRatio = 0x1p-13f;

// One build (a single problem or a batch) in either precision.  db/dc/dd are device
// arrays holding every problem's coefficients at its RootDesc::coef offset.  H[p] is the
// handle of problem p (allocated by the caller).  Per problem, code[p] is 0 or
// GM_ESINGULAR and growth[p] the block-pivoting growth flag of a mixed build.
int run_build(const gm_opts &o, double tol, const std::shared_ptr<DevPlan> &dpp, const double *db, const double *dc,
              const double *dd, std::vector<gm_handle *> &H, std::vector<int> &code, std::vector<int> &growth,
              const Tune &tu = Tune(), cudaGraph_t *record = nullptr) {
    const auto t_enter = std::chrono::steady_clock::now();
    std::vector<double> stamps;  // host time (ms) at the end of each phase, reported under GM_DEBUG
    auto stamp = [&] {
        if (debug_on())
            stamps.push_back(std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_enter).count());
    };
    const DevPlan &dp = *dpp;
    const Plan &P = dp.plan;
    cudaStream_t s = (cudaStream_t)o.stream;
    const bool mixed = o.precision == GM_PREC_MIXED;
    const bool blockpiv = mixed && o.pivoting != GM_PIVOT_PARTIAL;
    const int nb = o.panel_width > 0 ? o.panel_width : 16;  // measured best for both paths (n = 256, 512)
    if (nb > GJ_MAX_NB) return GM_EINVAL;
    const int split = o.split_digits ? o.split_digits : 6;
    if (mixed && (split < 3 || split > 6)) return GM_EINVAL;
    if (leaf_smem_bytes(dp.max_leaf_a, dp.max_leaf_b) > 220 * 1024) return GM_EUNSUPPORTED;
    if (mixed && std::max(mx_leaf_smem_bytes(dp.max_leaf_a, dp.max_leaf_b),
                          mx_leaf_lines_smem_bytes(dp.max_leaf_a, dp.max_leaf_b)) > 220 * 1024)
        return GM_EUNSUPPORTED;
    // the leaf kernel gives each inner-ring right-hand side one of 64 thread columns
    if (2 * (dp.max_leaf_a - 2) + 2 * (dp.max_leaf_b - 2) - 4 > 64) return GM_EUNSUPPORTED;
    if (mixed && !blockpiv) {
        int mm = P.r_root;
        for (const DevStage &ds : dp.stages) mm = std::max(mm, ds.max_m);
        if ((size_t)mm * nb * sizeof(float) > 200 * 1024) return GM_EUNSUPPORTED;
    }
    if (o.keep_levels && H.size() != 1) return GM_EUNSUPPORTED;
    for (gm_handle *h : H) {
        h->plan = dpp;
        h->L = P.L;
        h->split = split;
        h->kept_df32 = mixed;
    }
    int rc;
    int hbs_merges = 0, hbs_rank = 0, hbs_lr_rank = 0, hbs_fallbacks = 0;
    const size_t np = H.size();
    // declared ahead of every buffer: the capture ends before the look-ahead streams go
    LookAhead la;
    CaptureGuard cg;
    if (record) {  // record every launch of this build into a graph (nothing runs now)
        if (tol > 0.0 || o.keep_levels || o.timing) return GM_EINVAL;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        cg.s = s;
        cg.active = true;
    }
    DBuf stat;
    if ((rc = stat.alloc(np * sizeof(Status), s))) return rc;
    std::vector<Status> hst(np, Status{0, -1, 0x7ff0000000000000ull, 0, 0u});
    if (record) {
        k_status_init<<<(int)((np + 127) / 128), 128, 0, s>>>(stat.as<Status>(), (int)np);
        CK(cudaGetLastError());
    } else {
        CK(cudaMemcpyAsync(stat.p, hst.data(), np * sizeof(Status), cudaMemcpyHostToDevice, s));
    }
    Status *dst = stat.as<Status>();
    if (record) tl_recorded_status = dst;
    KTimer kt;
    kt.on = o.timing != 0;
    if (o.timing_mask) kt.mask = (unsigned)o.timing_mask;
    // 0: the default bound; a negative limit gives up at the first wait (tests the path)
    const int wait_limit = o.wait_limit != 0 ? o.wait_limit : (1 << 22);

    // the arena: FP64, or double-float pairs (same 8 bytes per element)
    DBuf arena_buf;
    void *arena = nullptr;
    const size_t arena_bytes = (size_t)P.arena_doubles * 8;
    if (o.keep_levels) {
        if (lib_malloc(&arena, arena_bytes ? arena_bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return GM_ENOMEM;
        }
        H[0]->kept_bufs.push_back(arena);
        for (size_t i = 0; i < P.leaves.size(); ++i)
            H[0]->kept.push_back({P.leaf_boxes[i], (char *)arena + P.leaves[i].off * 8});
        for (const Stage &st : P.stages)
            for (size_t i = 0; i < st.merges.size(); ++i)
                H[0]->kept.push_back({st.out_boxes[i], (char *)arena + st.merges[i].out * 8});
    } else {
        if ((rc = arena_buf.alloc(arena_bytes, s))) return rc;
        arena = arena_buf.p;
    }
    double *A64 = (double *)arena;
    float2 *Adf = (float2 *)arena;
    int64_t peak = arena_bytes;

    // leaves (Section 3.3 step 2)
    if (!mixed) {
        CK(launch_leaf(dp.d_leaves, P.leaves, dp.max_leaf_a, dp.max_leaf_b, db, dc, dd, A64, dst, 0, s, kt));
    } else {
        CK(mx_leaf(dp.d_leaves, P.leaves, dp.max_leaf_a, dp.max_leaf_b, db, dc, dd, Adf, dst, 0, s, kt));
    }

    // scratch of the sweeps, sized for the largest stage and for the roots
    int max_nm = (int)P.roots.size(), piv_ld = P.r_root;
    int64_t max_rows = 0, max_cols = 0, max_plane = 16, max_exp = 1, max_u12 = 0;
    for (const SysDesc &r : dp.h_root_sys) {
        max_rows += r.m;
        max_cols += r.ncol;
    }
    max_u12 = (int64_t)max_nm * nb * dp.max_root_ncol;
    for (size_t si = 0; si < dp.stages.size(); ++si) {
        const DevStage &ds = dp.stages[si];
        max_nm = std::max(max_nm, ds.nm);
        piv_ld = std::max(piv_ld, ds.max_m);
        max_rows = std::max<int64_t>(max_rows, ds.sum_rows);
        max_cols = std::max<int64_t>(max_cols, ds.sum_cols);
        max_plane = std::max<int64_t>(max_plane, ds.dig_elems);
        max_exp = std::max<int64_t>(max_exp, ds.exp_elems);
        max_u12 = std::max<int64_t>(max_u12, (int64_t)ds.nm * nb * ds.max_ncol);
    }
    DBuf piv, u12;                                          // FP64 sweep
    DBuf perm, perm_n, a11, fdig, rdig, fex, rex;           // mixed, partial pivoting
    DBuf ydig, xdig, yex, xex;                              // mixed Schur updates
    DBuf bxd, bad, bxe, bae, bpmag, bfdig, bfex, brdig, brex;  // mixed, block pivoting
    MxScratch scr;
    BlkScratch bscr;
    // on every exit: nothing on the look-ahead streams may still read the scratch buffers
    // above when they are released (early returns); a build being recorded ran nothing
    struct StreamsIdle {
        LookAhead &la;
        const CaptureGuard &cg;
        ~StreamsIdle() {
            if (cg.active) return;
            if (la.s1) cudaStreamSynchronize(la.s1);
            if (la.s2) cudaStreamSynchronize(la.s2);
            if (la.s3) cudaStreamSynchronize(la.s3);
        }
    } idle{la, cg};
    if (!mixed) {
        if ((rc = piv.alloc((size_t)max_nm * piv_ld * sizeof(int), s))) return rc;
        if ((rc = u12.alloc((size_t)max_u12 * 8, s))) return rc;
    } else {
        if ((rc = ydig.alloc((size_t)split * max_plane * 2, s)) || (rc = xdig.alloc((size_t)split * max_plane * 2, s)) ||
            (rc = yex.alloc((size_t)max_exp * sizeof(int), s)) || (rc = xex.alloc((size_t)max_exp * sizeof(int), s)))
            return rc;
        if (blockpiv) {
            const size_t sq = (size_t)max_nm * 64;
            // two factor output sets (the early-factor schedule alternates between them)
            if ((rc = bxd.alloc(2 * (size_t)split * sq * 64 * 2, s)) ||
                (rc = bad.alloc(2 * (size_t)split * sq * 64 * 2, s)) || (rc = bxe.alloc(2 * sq * sizeof(int), s)) ||
                (rc = bae.alloc(2 * sq * sizeof(int), s)) || (rc = bpmag.alloc(2 * sq * sizeof(float), s)) ||
                (rc = bfdig.alloc(2 * (size_t)split * max_rows * 64 * 2, s)) ||
                (rc = bfex.alloc(2 * (size_t)max_rows * sizeof(int), s)) ||
                (rc = brdig.alloc(2 * (size_t)split * max_cols * 64 * 2, s)) ||
                (rc = brex.alloc(2 * (size_t)max_cols * sizeof(int), s)))
                return rc;
            bscr.x_dig = bxd.as<__nv_bfloat16>();
            bscr.a11_dig = bad.as<__nv_bfloat16>();
            bscr.x_ex = bxe.as<int>();
            bscr.a11_ex = bae.as<int>();
            bscr.pmag = bpmag.as<float>();
            bscr.x_dig2 = bscr.x_dig + (size_t)split * sq * 64;
            bscr.a11_dig2 = bscr.a11_dig + (size_t)split * sq * 64;
            bscr.x_ex2 = bscr.x_ex + sq;
            bscr.a11_ex2 = bscr.a11_ex + sq;
            bscr.pmag2 = bscr.pmag + sq;
            for (int q = 0; q < 2; ++q) {
                bscr.fdig[q] = bfdig.as<__nv_bfloat16>() + (size_t)q * split * max_rows * 64;
                bscr.fex[q] = bfex.as<int>() + (size_t)q * max_rows;
                bscr.rdig[q] = brdig.as<__nv_bfloat16>() + (size_t)q * split * max_cols * 64;
                bscr.rex[q] = brex.as<int>() + (size_t)q * max_cols;
            }
            if (!la.create(o.background != 0)) return GM_ECUDA;
            bscr.wait_limit = wait_limit;
            bscr.rtile32_max = tu.rtile32_max;
            bscr.early = tu.early != 0;
            bscr.upd_tiles = tu.upd_tiles;
            bscr.a11first = tu.a11 != 0;
            bscr.sms = device_sms();
            bscr.s3 = la.s3;
            bscr.ev_rr = la.d;
            bscr.ev_next = la.e;
            bscr.ev_rest2[0] = la.f[0];
            bscr.ev_rest2[1] = la.f[1];
            bscr.s1 = la.s1;
            bscr.s2 = la.s2;
            bscr.ev_r = la.a;
            bscr.ev_rest = la.b;
            bscr.ev_join = la.c;
        } else {
            if ((rc = perm.alloc((size_t)max_nm * 4 * GJ_MAX_NB * sizeof(int), s)) ||
                (rc = perm_n.alloc((size_t)max_nm * sizeof(int), s)) ||
                (rc = a11.alloc((size_t)max_nm * GJ_MAX_NB * GJ_MAX_NB * sizeof(float2), s)) ||
                (rc = fdig.alloc((size_t)split * max_rows * 16 * 2, s)) ||
                (rc = rdig.alloc((size_t)split * max_cols * 16 * 2, s)) ||
                (rc = fex.alloc((size_t)max_rows * sizeof(int), s)) ||
                (rc = rex.alloc((size_t)max_cols * sizeof(int), s)))
                return rc;
            scr.perm = perm.as<int>();
            scr.perm_n = perm_n.as<int>();
            scr.a11inv = a11.as<float2>();
            scr.fdig = fdig.as<__nv_bfloat16>();
            scr.rdig = rdig.as<__nv_bfloat16>();
            scr.fex = fex.as<int>();
            scr.rex = rex.as<int>();
        }
    }
    // one dense sweep over a set of systems: FP64 Gauss-Jordan, or a mixed sweep
    auto sweep = [&](const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol, void *ws,
                     int sum_rows, int sum_cols, int stage) -> cudaError_t {
        if (!mixed)
            return launch_gj_sweep(d_sys, h_sys, max_m, max_ncol, (double *)ws, nb, piv.as<int>(), piv_ld,
                                   u12.as<double>(), (int64_t)nb * max_ncol, dst, stage, s, kt);
        if (blockpiv) {
            bscr.inv_plane = (int64_t)h_sys.size() * 64 * 64;
            bscr.fplane = (int64_t)sum_rows * 64;
            bscr.cplane = (int64_t)sum_cols * 64;
            return blk_gj_sweep(d_sys, h_sys, max_m, max_ncol, (float2 *)ws, split, bscr, dst, stage, s, kt);
        }
        scr.fplane = (int64_t)sum_rows * 16;
        scr.rplane = (int64_t)sum_cols * 16;
        return mx_gj_sweep(d_sys, h_sys, max_m, max_ncol, (float2 *)ws, nb, split, scr, dst, stage, s, kt);
    };

    stamp();
    // merge stages (Section 3.3 step 3): per level, horizontal then vertical
    for (size_t si = 0; si < dp.stages.size(); ++si) {
        const DevStage &ds = dp.stages[si];
        const Stage &hs = P.stages[si];
        if (ds.nm == 0) continue;
        DBuf ws;
        if ((rc = ws.alloc(ds.ws_doubles * 8, s))) return rc;
        peak = std::max(peak, (int64_t)(arena_bytes + ds.ws_doubles * 8));
        if (!mixed) {
            CK(launch_merge_assemble(ds.d_merges, ds.nm, ds.d_tab, A64, ws.as<double>(), ds.max_elems, db, dc, dd, 0,
                                     s, kt));
            // tol > 0: merges whose shared edge has at least hbs_min_edge nodes solve their
            // interface system by the accelerated Step 1 (HBS inverses of S33 and of its
            // Schur complement); the others, and any whose ranks exceed the cap, stay dense
            std::vector<SysDesc> dense;
            std::vector<int> hbs_idx;  // merges of this stage solved by the accelerated merge
            bool any_hbs = false;
            std::vector<int> cand;     // merges that try the accelerated Step 1
            for (int i = 0; i < ds.nm; ++i) {
                const MergeDesc &md = hs.merges[i];
                if (tol > 0.0 && md.sp + 2 >= o.hbs_min_edge && md.sp > o.hbs_leaf) cand.push_back(i);
            }
            std::vector<int> crc(cand.size(), GM_OK);
            if (cand.size() > 1 && !kt.on) {
                // the merges are independent and each factorisation is a chain of small
                // launches and host synchronisations: run them side by side
                std::vector<int> rk(cand.size(), 0);
                std::vector<double> fl(cand.size(), 0.0);
                std::vector<std::map<std::pair<int, int>, int>> hints(cand.size());
                hbs_hints_freeze();
                rc = run_lanes((int)cand.size(), s, [&](int j, cudaStream_t ls) {
                    const MergeDesc &md = hs.merges[cand[j]];
                    hbs_hints_record(&hints[j]);
                    hbs_flops_take();
                    crc[j] = hbs_block_solve(ws.as<double>() + ds.h_sys[cand[j]].off, md.sp, md.rp, o.hbs_leaf,
                                             tol, ls, &rk[j]);
                    fl[j] = hbs_flops_take();
                    hbs_hints_record(nullptr);
                });
                hbs_hints_thaw(hints);
                if (rc) return rc;
                for (size_t j = 0; j < cand.size(); ++j) {
                    hbs_rank = std::max(hbs_rank, rk[j]);
                    kt.flops[GM_K_PANEL] += fl[j];
                    kt.launches[GM_K_PANEL] += 1;
                }
            } else {
                for (size_t j = 0; j < cand.size(); ++j) {
                    const MergeDesc &md = hs.merges[cand[j]];
                    hbs_flops_take();
                    kt.begin(GM_K_PANEL, 0.0, s);
                    crc[j] = hbs_block_solve(ws.as<double>() + ds.h_sys[cand[j]].off, md.sp, md.rp, o.hbs_leaf, tol,
                                             s, &hbs_rank);
                    kt.end(s);
                    kt.flops[GM_K_PANEL] += hbs_flops_take();
                }
            }
            for (int i = 0, j = 0; i < ds.nm; ++i) {
                if (j < (int)cand.size() && cand[j] == i) {
                    const int r2 = crc[j++];
                    if (r2 == GM_OK) {
                        ++hbs_merges;
                        any_hbs = true;
                        hbs_idx.push_back(i);
                        continue;
                    }
                    if (r2 != GM_EUNSUPPORTED && r2 != HBS_UNSTABLE) return r2;
                    ++hbs_fallbacks;
                }
                dense.push_back(ds.h_sys[i]);
            }
            if (!any_hbs) {
                CK(sweep(ds.d_sys, ds.h_sys, ds.max_m, ds.max_ncol, ws.p, ds.sum_rows, ds.sum_cols, (int)si + 1));
            } else if (!dense.empty()) {
                int ro = 0, co = 0, mm = 0, mc = 0;
                for (SysDesc &q : dense) {
                    q.roff = ro;
                    q.coff = co;
                    ro += q.m;
                    co += q.ncol;
                    mm = std::max(mm, q.m);
                    mc = std::max(mc, q.ncol);
                }
                DBuf dsub;
                if ((rc = dsub.alloc(dense.size() * sizeof(SysDesc), s))) return rc;
                CK(cudaMemcpyAsync(dsub.p, dense.data(), dense.size() * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
                CK(sweep(dsub.as<SysDesc>(), dense, mm, mc, ws.p, ro, co, (int)si + 1));
            }
            if (hbs_idx.empty()) {
                CK(launch_merge_update(ds.d_merges, hs.merges, ds.d_tab, A64, ws.as<double>(), A64, ds.max_rp, db, dc,
                                       dd, 0, s, kt));
            } else {
                // Steps 2-3 of the accelerated merge for the merges solved by Step 1: S13,
                // S24 compressed, the update in factored form; the others as usual
                std::vector<MergeDesc> dm;
                for (int i = 0, j = 0; i < ds.nm; ++i) {
                    if (j < (int)hbs_idx.size() && hbs_idx[j] == i) {
                        ++j;
                        continue;
                    }
                    dm.push_back(hs.merges[i]);
                }
                if (!dm.empty()) {
                    DBuf dsub;
                    if ((rc = dsub.alloc(dm.size() * sizeof(MergeDesc), s))) return rc;
                    CK(cudaMemcpyAsync(dsub.p, dm.data(), dm.size() * sizeof(MergeDesc), cudaMemcpyHostToDevice, s));
                    int mrp = 0;
                    for (const MergeDesc &q : dm) mrp = std::max(mrp, q.rp);
                    CK(launch_merge_update(dsub.as<MergeDesc>(), dm, ds.d_tab, A64, ws.as<double>(), A64, mrp, db, dc,
                                           dd, 0, s, kt));
                }
                if (hbs_idx.size() > 1 && !kt.on) {  // side by side, like Step 1
                    const size_t nh = hbs_idx.size();
                    std::vector<int> lrc(nh, GM_OK), rk(nh, 0);
                    std::vector<double> fl(nh, 0.0);
                    std::vector<std::map<std::pair<int, int>, int>> hints(nh);
                    hbs_hints_freeze();
                    rc = run_lanes((int)nh, s, [&](int j, cudaStream_t ls) {
                        const int i = hbs_idx[j];
                        KTimer lkt;  // untimed: only its flop count is kept
                        hbs_hints_record(&hints[j]);
                        hbs_flops_take();
                        lrc[j] = hbs_merge_lowrank(hs.merges[i], ds.d_merges + i, ds.d_tab, A64,
                                                   ws.as<double>() + ds.h_sys[i].off, A64, db, dc, dd, tol, ls, lkt,
                                                   &rk[j]);
                        fl[j] = hbs_flops_take() + lkt.flops[GM_K_MERGEUPDATE];
                        hbs_hints_record(nullptr);
                    });
                    hbs_hints_thaw(hints);
                    if (rc) return rc;
                    for (size_t j = 0; j < nh; ++j) {
                        if (lrc[j]) return lrc[j];
                        hbs_lr_rank = std::max(hbs_lr_rank, rk[j]);
                        kt.flops[GM_K_MERGEUPDATE] += fl[j];
                        kt.launches[GM_K_MERGEUPDATE] += 1;
                    }
                } else {
                    for (int i : hbs_idx) {
                        hbs_flops_take();
                        if ((rc = hbs_merge_lowrank(hs.merges[i], ds.d_merges + i, ds.d_tab, A64,
                                                    ws.as<double>() + ds.h_sys[i].off, A64, db, dc, dd, tol, s, kt,
                                                    &hbs_lr_rank)))
                            return rc;
                        kt.flops[GM_K_MERGEUPDATE] += hbs_flops_take();
                    }
                }
            }
        } else {
            CK(mx_merge_assemble(ds.d_merges, ds.nm, ds.d_tab, Adf, ws.as<float2>(), ds.max_elems, db, dc, dd, 0, s,
                                 kt));
            CK(sweep(ds.d_sys, ds.h_sys, ds.max_m, ds.max_ncol, ws.p, ds.sum_rows, ds.sum_cols, (int)si + 1));
            CK(mx_merge_update(ds.d_merges, hs.merges, ds.d_tab, Adf, ws.as<float2>(), Adf, ds.max_rp, split,
                               ydig.as<__nv_bfloat16>(), yex.as<int>(), xdig.as<__nv_bfloat16>(), xex.as<int>(),
                               ds.dig_elems, db, dc, dd, 0, dst, s, kt, wait_limit, tu.tc_min_k));
        }
        stamp();
    }

    DBuf rws;
    // roots eliminated densely: all of them, or with tol > 0 those whose HBS inverse
    // failed its residual check
    std::vector<int> dense_roots;
    if (tol > 0.0) {
        // HBS roots (Sections 4-5): compress every S_root and invert it by Algorithm 1;
        // the solve applies Algorithm 2 (no dense T)
        hbs_flops_take();
        kt.begin(GM_K_ROOT, 0.0, s);
        for (size_t i = 0; i < P.roots.size(); ++i) {
            const RootDesc &r = P.roots[i];
            gm_handle *h = H[r.problem];
            const double *S64 = A64 + r.off;
            DBuf conv;
            if (mixed) {
                if ((rc = conv.alloc((size_t)r.r * r.r * 8, s))) return rc;
                CK(hbs_df32_to_f64(Adf + r.off, conv.as<double>(), (int64_t)r.r * r.r, s));
                S64 = conv.as<double>();
            }
            h->hbs = new HbsRoot();
            rc = hbs_build_root(S64, r.r, r.n, o.hbs_leaf, tol, db + r.coef, dc + r.coef, dd + r.coef, s, *h->hbs);
            if (rc == HBS_UNSTABLE) {  // Algorithm 1 unstable here: a dense root instead
                hbs_free(*h->hbs);
                delete h->hbs;
                h->hbs = nullptr;
                dense_roots.push_back((int)i);
                ++hbs_fallbacks;
                continue;
            }
            if (rc) return rc;
            peak = std::max(peak, (int64_t)(arena_bytes + h->hbs->pool_doubles * 8));
        }
        kt.end(s);
        kt.flops[GM_K_ROOT] += hbs_flops_take();
    } else {
        for (size_t i = 0; i < P.roots.size(); ++i) dense_roots.push_back((int)i);
    }
    if (!dense_roots.empty()) {
    // roots (Section 3.3 step 4): X = S_root^{-1} B for every problem in one sweep
    if ((rc = rws.alloc(dp.root_ws * 8, s))) return rc;
    peak = std::max(peak, (int64_t)(arena_bytes + dp.root_ws * 8));
    int max_r = 0, max_c = 0, sum_rr = 0, sum_rc = 0;
    std::vector<SysDesc> rsys;
    for (int i : dense_roots) {
        const RootDesc &r = P.roots[i];
        SysDesc sy = dp.h_root_sys[i];
        sy.roff = sum_rr;
        sy.coff = sum_rc;
        rsys.push_back(sy);
        max_r = std::max(max_r, r.r);
        max_c = std::max(max_c, sy.ncol);
        sum_rr += sy.m;
        sum_rc += sy.ncol;
        if (!mixed)
            CK(launch_root_assemble(A64 + r.off, r.r, r.n, rws.as<double>() + sy.off, db + r.coef, dc + r.coef,
                                    dd + r.coef, s, kt));
        else
            CK(mx_root_assemble(Adf + r.off, r.r, r.n, rws.as<float2>() + sy.off, db + r.coef, dc + r.coef,
                                dd + r.coef, s, kt));
    }
    if (dense_roots.size() == P.roots.size()) {
        CK(sweep(dp.d_root_sys, dp.h_root_sys, max_r, dp.max_root_ncol, rws.p, sum_rr, sum_rc,
                 (int)dp.stages.size() + 1));
    } else {  // a subset: descriptors with their own row and column offsets
        DBuf dsub;
        if ((rc = dsub.alloc(rsys.size() * sizeof(SysDesc), s))) return rc;
        CK(cudaMemcpyAsync(dsub.p, rsys.data(), rsys.size() * sizeof(SysDesc), cudaMemcpyHostToDevice, s));
        CK(sweep(dsub.as<SysDesc>(), rsys, max_r, max_c, rws.p, sum_rr, sum_rc, (int)dp.stages.size() + 1));
    }
    stamp();
    for (int i : dense_roots) {
        const RootDesc &r = P.roots[i];
        gm_handle *h = H[r.problem];
        const int nb4 = 4 * r.n;
        const SysDesc &sy = dp.h_root_sys[i];
        if (lib_malloc((void **)&h->T, (size_t)nb4 * nb4 * 8) != cudaSuccess) {
            cudaGetLastError();
            return GM_ENOMEM;
        }
        if (!mixed) {
            CK(launch_root_finalize(rws.as<double>() + sy.off, r.r, r.n, h->T, s, kt));
        } else {
            const int kpadT = mx_kpad(nb4);
            if (lib_malloc((void **)&h->Tdf, (size_t)nb4 * nb4 * sizeof(float2)) != cudaSuccess ||
                lib_malloc((void **)&h->tdig, (size_t)split * nb4 * kpadT * 2) != cudaSuccess ||
                lib_malloc((void **)&h->tex, (size_t)nb4 * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return GM_ENOMEM;
            }
            CK(mx_root_finalize(rws.as<float2>() + sy.off, r.r, r.n, h->T, h->Tdf, h->tdig, h->tex, split,
                                stat.as<Status>() + r.problem, (int)dp.stages.size() + 1, s, kt));
        }
    }
    stamp();
    }
    if (record) {
        cg.active = false;
        CK(cudaStreamEndCapture(s, record));
        return GM_OK;
    }
    CK(cudaMemcpyAsync(hst.data(), stat.p, np * sizeof(Status), cudaMemcpyDeviceToHost, s));
    // release temporaries (stream-ordered) before the final synchronisation
    for (DBuf *b : {&rws, &piv, &u12, &perm, &perm_n, &a11, &fdig, &rdig, &fex, &rex, &ydig, &xdig, &yex, &xex, &bxd,
                    &bad, &bxe, &bae, &bpmag, &bfdig, &bfex, &brdig, &brex, &arena_buf, &stat})
        b->release();
    const auto t_enq = std::chrono::steady_clock::now();
    CK(cudaStreamSynchronize(s));
    if (debug_on()) {  // host time to enqueue the build, and until it finished on the device
        const auto t_done = std::chrono::steady_clock::now();
        fprintf(stderr, "gm: build enqueued in %.3f ms, done after %.3f ms; phases end at",
                std::chrono::duration<double, std::milli>(t_enq - t_enter).count(),
                std::chrono::duration<double, std::milli>(t_done - t_enter).count());
        for (double x : stamps) fprintf(stderr, " %.2f", x);
        fprintf(stderr, " ms\n");
    }
    int launches = 0;
    gm_info_t info{};
    for (int f = 0; f < GM_K_NFAM; ++f) {
        launches += kt.launches[f];
        info.kernel_launches[f] = kt.launches[f];
        info.kernel_flops[f] = kt.flops[f];
    }
    kt.collect(info.kernel_ms);
    info.launches = launches;
    info.peak_workspace = peak;
    info.pivoting = blockpiv ? GM_PIVOT_BLOCK : GM_PIVOT_PARTIAL;
    info.levels = P.L_user;
    info.precision = o.precision;
    info.load_rank = -1;
    code.assign(np, 0);
    growth.assign(np, 0);
    int first = GM_OK;
    for (size_t p = 0; p < np; ++p) {
        gm_handle *h = H[p];
        const Status &st = hst[p];
        double mp;
        memcpy(&mp, &st.min_piv, 8);
        gm_info_t hi = info;
        hi.n = h->n;
        hi.leaf = h->leaf;
        hi.dtn_bytes = h->hbs ? 0 : (long long)16 * h->n * h->n * 8;
        hi.hbs_merges = hbs_merges;
        hi.hbs_max_rank = hbs_rank;
        hi.hbs_update_rank = hbs_lr_rank;
        hi.hbs_fallbacks = hbs_fallbacks;
        if (h->hbs) {
            hi.hbs_levels = h->hbs->L;
            hi.hbs_max_rank = std::max(hbs_rank, h->hbs->max_rank);
            hi.hbs_bytes = h->hbs->pool_doubles * 8;
            hi.hbs_operator_bytes = hbs_operator_doubles(*h->hbs) * 8;
            hi.resident_bytes = hi.hbs_bytes;
        } else {
            const long long N = 4LL * h->n;
            hi.resident_bytes = N * N * 8;
            if (mixed) hi.resident_bytes += N * N * 8 + (long long)split * N * mx_kpad((int)N) * 2 + N * 4;
        }
        hi.min_pivot_ratio = mp / (4.0 * (h->n + 1.0) * (h->n + 1.0));
        hi.bad_stage = st.code ? st.where : -1;
        float rho;
        memcpy(&rho, &st.rho, 4);
        hi.refine_ratio = blockpiv ? (double)rho : 0.0;
        h->info = hi;
        code[p] = st.code;
        // a refinement ratio rho leaves an error near rho^2 per block solve
        growth[p] = st.growth || (blockpiv && !(rho <= kMaxRefineRatio));
        if (st.code && first == GM_OK) first = st.code;
    }
    return first;
}

gm_handle *new_handle(const std::pair<int, int> &p, int precision) {
    gm_handle *h = new gm_handle();
    h->n = p.first;
    h->leaf = p.second;
    h->precision = precision;
    return h;
}

// Largest reaction coefficient of each problem (coefficients concatenated, problem p at
// off[p]): per-block maxima, reduced on the host.
__global__ void k_max_d(const double *__restrict__ d, const int64_t *__restrict__ off, double *__restrict__ part) {
    const int p = blockIdx.y;
    const int64_t lo = off[p], hi = off[p + 1];
    double v = -1e300;
    for (int64_t e = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < hi; e += (int64_t)gridDim.x * blockDim.x)
        v = fmax(v, d[e]);
    __shared__ double sm[256];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)p * gridDim.x + blockIdx.x] = sm[0];
}

int max_reaction(const std::vector<std::pair<int, int>> &probs, const double *dd, cudaStream_t s,
                 std::vector<double> &maxd) {
    const int np = (int)probs.size(), nb = 32;
    std::vector<int64_t> off(np + 1, 0);
    for (int p = 0; p < np; ++p) off[p + 1] = off[p] + (int64_t)probs[p].first * probs[p].first;
    DBuf doff, part;
    int rc;
    if ((rc = doff.alloc(off.size() * 8, s)) || (rc = part.alloc((size_t)np * nb * 8, s))) return rc;
    CK(cudaMemcpyAsync(doff.p, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s));
    k_max_d<<<dim3(nb, np), 256, 0, s>>>(dd, doff.as<int64_t>(), part.as<double>());
    CK(cudaGetLastError());
    std::vector<double> h((size_t)np * nb);
    CK(cudaMemcpyAsync(h.data(), part.p, h.size() * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    maxd.assign(np, -1e300);
    for (int p = 0; p < np; ++p)
        for (int b = 0; b < nb; ++b) maxd[p] = std::max(maxd[p], h[(size_t)p * nb + b]);
    return GM_OK;
}

// Build the problems listed in `sub` (indices into probs; coefficients of problem p at
// off[p] of db/dc/dd) as one batch with options o; Hs receives their handles.
// ----------------------------------------------------------------------------- tuning, graphs

// Builds are tuned and recorded per plan and per option that changes what is launched.
using TuneKey = std::tuple<const DevPlan *, int, int, int, int, int, int>;
TuneKey tune_key(const std::shared_ptr<DevPlan> &dp, const gm_opts &o) {
    return TuneKey(dp.get(), o.precision, o.pivoting, o.split_digits, o.panel_width, o.wait_limit, o.background);
}
std::mutex g_tune_mu;
std::map<TuneKey, Tune> g_tunes;

bool find_tune(const TuneKey &k, Tune &t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tunes.find(k);
    if (it == g_tunes.end()) return false;
    t = it->second;
    return true;
}
void store_tune(const TuneKey &k, const Tune &t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tunes[k] = t;
}

// The autotuner: whole builds of the plan timed on the host (each ends with a stream
// synchronisation), best of two per candidate, one launch-shape parameter at a time --
// the R kernel's 32-column tiles (never / while the step leaves SMs idle / always), then
// the merge update's tcgen05 bound on the interface length (192, 448, never).
int autotune(const gm_opts &o, const std::shared_ptr<DevPlan> &dp, const std::vector<std::pair<int, int>> &keys,
             const double *sb, const double *sc, const double *sd, Tune &best) {
    auto time_of = [&](const Tune &t) -> double {
        double bt = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            std::vector<gm_handle *> Hs;
            for (const auto &k : keys) Hs.push_back(new_handle(k, o.precision));
            std::vector<int> code, growth;
            const auto t0 = std::chrono::steady_clock::now();
            const int rc = run_build(o, 0.0, dp, sb, sc, sd, Hs, code, growth, t);
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            for (gm_handle *h : Hs) gm_free(h);
            if (rc != GM_OK) return 1e300;
            bt = std::min(bt, ms);
        }
        if (debug_on())
            fprintf(stderr, "gm: autotune rtile32_max %d early %d a11 %d tc_min_k %d upd_tiles %d: %.3f ms\n",
                    t.rtile32_max, t.early, t.a11, t.tc_min_k, t.upd_tiles, bt);
        return bt;
    };
    best = Tune();
    double tb = time_of(best);
    if (tb >= 1e300) return GM_OK;  // the plan does not build cleanly as is: keep the defaults
    for (int r : {0, 1 << 30}) {
        Tune t = best;
        t.rtile32_max = r;
        const double x = time_of(t);
        if (x < tb) {
            tb = x;
            best = t;
        }
    }
    if (o.precision == GM_PREC_MIXED)
        for (int u : {0, 2, 4, -1}) {
            if (u == best.upd_tiles) continue;
            Tune t = best;
            t.upd_tiles = u;
            const double x = time_of(t);
            if (x < tb) {
                tb = x;
                best = t;
            }
        }
    if (o.precision == GM_PREC_MIXED) {
        Tune t = best;
        t.a11 = !best.a11;
        const double x = time_of(t);
        if (x < tb) {
            tb = x;
            best = t;
        }
    }
    if (o.precision == GM_PREC_MIXED) {
        Tune t = best;
        t.early = !best.early;
        const double x = time_of(t);
        if (x < tb) {
            tb = x;
            best = t;
        }
    }
    if (o.precision == GM_PREC_MIXED)
        for (int k : {448, 1 << 30}) {
            Tune t = best;
            t.tc_min_k = k;
            const double x = time_of(t);
            if (x < tb) {
                tb = x;
                best = t;
            }
        }
    return GM_OK;
}

// A build recorded into a CUDA graph, with every buffer it reads or writes.
struct GraphEntry {
    TuneKey key;
    Tune tune;
    std::shared_ptr<DevPlan> plan;
    char *mem = nullptr;  // coefficient staging, then everything the build allocated, in order
    cudaGraphExec_t exec = nullptr;
    double *cb = nullptr, *cc = nullptr, *cd = nullptr;
    int64_t total = 0;
    Status *stat = nullptr;
    struct Out {
        size_t T = 0, Tdf = 0, tdig = 0, tex = 0;  // offsets in mem (0: none)
        size_t nT = 0, nTdf = 0, ntdig = 0, ntex = 0;
    };
    std::vector<Out> outs;
    std::vector<gm_info_t> info;  // per problem: what does not depend on the run's status
    long long last_use = 0;
    ~GraphEntry() {
        if (exec) cudaGraphExecDestroy(exec);
        if (mem) cudaFree(mem);
    }
};
std::mutex g_graph_mu;
std::vector<std::shared_ptr<GraphEntry>> g_graphs;
long long g_graph_tick = 0;
constexpr size_t kMaxGraphs = 8;
std::shared_ptr<GraphEntry> find_graph(const TuneKey &k, const Tune &t) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto &e : g_graphs)
        if (e->key == k && e->tune.rtile32_max == t.rtile32_max && e->tune.tc_min_k == t.tc_min_k &&
            e->tune.early == t.early && e->tune.upd_tiles == t.upd_tiles && e->tune.a11 == t.a11) {
            e->last_use = ++g_graph_tick;
            return e;
        }
    return nullptr;
}

// Record the plan's build into a graph with buffers of its own (`bytes` summed over the
// first build's allocations).  Failure only means later builds run as usual.
void record_graph(const gm_opts &o, double tol, const std::shared_ptr<DevPlan> &dp,
                  const std::vector<std::pair<int, int>> &keys, int64_t total, const Tune &tu, const TuneKey &tk,
                  size_t bytes, const std::vector<gm_handle *> &built) {
    auto E = std::make_shared<GraphEntry>();
    E->key = tk;
    E->tune = tu;
    E->plan = dp;
    E->total = total;
    const size_t coef = BumpCtx::align(3 * (size_t)total * sizeof(double));
    if (cudaMalloc((void **)&E->mem, coef + bytes + 4096) != cudaSuccess) {
        cudaGetLastError();
        E->mem = nullptr;
        return;
    }
    E->cb = (double *)E->mem;
    E->cc = E->cb + total;
    E->cd = E->cc + total;
    BumpCtx ctx;
    ctx.base = E->mem + coef;
    ctx.cap = bytes + 4096;
    std::vector<gm_handle *> Hd;
    for (const auto &k : keys) Hd.push_back(new_handle(k, o.precision));
    std::vector<int> code, growth;
    cudaGraph_t g = nullptr;
    tl_bump = &ctx;
    tl_recorded_status = nullptr;
    int rc = run_build(o, tol, dp, E->cb, E->cc, E->cd, Hd, code, growth, tu, &g);
    tl_bump = nullptr;
    E->stat = tl_recorded_status;
    // per-node priorities: the look-ahead's chain (high) and the rest of each update (low)
    // keep the priorities of the streams they were recorded from
    if (rc == GM_OK && g && E->stat &&
        cudaGraphInstantiateWithFlags(&E->exec, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess) {
        auto off = [&](const void *p) { return p ? (size_t)((const char *)p - E->mem) : (size_t)0; };
        for (size_t i = 0; i < Hd.size(); ++i) {
            gm_handle *h = Hd[i];
            GraphEntry::Out q;
            const size_t N = 4 * (size_t)h->n;
            q.T = off(h->T);
            q.nT = N * N * 8;
            if (h->Tdf) {
                q.Tdf = off(h->Tdf);
                q.nTdf = N * N * sizeof(float2);
                q.tdig = off(h->tdig);
                q.ntdig = (size_t)h->split * N * mx_kpad((int)N) * 2;
                q.tex = off(h->tex);
                q.ntex = N * sizeof(int);
            }
            E->outs.push_back(q);
            E->info.push_back(built[i]->info);
        }
    } else {
        cudaGetLastError();
        if (E->exec) cudaGraphExecDestroy(E->exec);
        E->exec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    for (gm_handle *h : Hd) {  // their buffers belong to the graph
        h->T = nullptr;
        h->Tdf = nullptr;
        h->tdig = nullptr;
        h->tex = nullptr;
        gm_free(h);
    }
    if (!E->exec) return;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    E->last_use = ++g_graph_tick;
    if (g_graphs.size() >= kMaxGraphs) {  // drop the least recently used
        auto v = std::min_element(g_graphs.begin(), g_graphs.end(),
                                  [](const auto &a, const auto &b) { return a->last_use < b->last_use; });
        g_graphs.erase(v);
    }
    g_graphs.push_back(E);
}

// A later build of a recorded plan: coefficients in, one graph launch, the operators out.
int replay(GraphEntry &E, const gm_opts &o, const std::vector<std::pair<int, int>> &keys, const double *sb,
           const double *sc, const double *sd, int64_t total, std::vector<gm_handle *> &Hs, std::vector<int> &code,
           std::vector<int> &growth) {
    cudaStream_t s = (cudaStream_t)o.stream;
    const size_t cb = (size_t)total * sizeof(double);
    CK(cudaMemcpyAsync(E.cb, sb, cb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(E.cc, sc, cb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(E.cd, sd, cb, cudaMemcpyDeviceToDevice, s));
    CK(cudaGraphLaunch(E.exec, s));
    const bool mixed = o.precision == GM_PREC_MIXED;
    const int split = o.split_digits ? o.split_digits : 6;
    for (size_t i = 0; i < keys.size(); ++i) {
        gm_handle *h = new_handle(keys[i], o.precision);
        Hs.push_back(h);
        h->plan = E.plan;
        h->L = E.plan->plan.L;
        h->split = split;
        h->kept_df32 = mixed;
        const GraphEntry::Out &q = E.outs[i];
        auto out = [&](void **dst, size_t offs, size_t n) -> int {
            if (!n) return GM_OK;
            if (lib_malloc(dst, n) != cudaSuccess) return GM_ENOMEM;
            return cudaMemcpyAsync(*dst, E.mem + offs, n, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? GM_OK
                                                                                                        : GM_ECUDA;
        };
        int rc;
        if ((rc = out((void **)&h->T, q.T, q.nT)) || (rc = out((void **)&h->Tdf, q.Tdf, q.nTdf)) ||
            (rc = out((void **)&h->tdig, q.tdig, q.ntdig)) || (rc = out((void **)&h->tex, q.tex, q.ntex)))
            return rc;
    }
    std::vector<Status> hst(keys.size());
    CK(cudaMemcpyAsync(hst.data(), E.stat, hst.size() * sizeof(Status), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const bool blockpiv = mixed && o.pivoting != GM_PIVOT_PARTIAL;
    code.assign(keys.size(), 0);
    growth.assign(keys.size(), 0);
    int first = GM_OK;
    for (size_t p = 0; p < keys.size(); ++p) {
        gm_handle *h = Hs[p];
        const Status &st = hst[p];
        double mp;
        memcpy(&mp, &st.min_piv, 8);
        gm_info_t hi = E.info[p];
        hi.min_pivot_ratio = mp / (4.0 * (h->n + 1.0) * (h->n + 1.0));
        hi.bad_stage = st.code ? st.where : -1;
        float rho;
        memcpy(&rho, &st.rho, 4);
        hi.refine_ratio = blockpiv ? (double)rho : 0.0;
        hi.pivot_fallback = 0;
        h->info = hi;
        code[p] = st.code;
        growth[p] = st.growth || (blockpiv && !(rho <= kMaxRefineRatio));
        if (st.code && first == GM_OK) first = st.code;
    }
    return first;
}

int build_subset(const gm_opts &o, double tol, const std::vector<std::pair<int, int>> &probs,
                 const std::vector<int64_t> &off, const std::vector<int> &sub, const double *db, const double *dc,
                 const double *dd, std::vector<gm_handle *> &Hs, std::vector<int> &code, std::vector<int> &growth) {
    cudaStream_t s = (cudaStream_t)o.stream;
    std::vector<std::pair<int, int>> keys;
    int64_t total = 0;
    for (int p : sub) {
        keys.push_back(probs[p]);
        total += (int64_t)probs[p].first * probs[p].first;
    }
    DBuf coef;
    const double *sb = db, *sc = dc, *sd = dd;
    int rc;
    if (sub.size() != probs.size()) {  // the subset's coefficients, concatenated in subset order
        if ((rc = coef.alloc(3 * (size_t)total * sizeof(double), s))) return rc;
        double *b2 = coef.as<double>(), *c2 = b2 + total, *d2 = c2 + total;
        int64_t at = 0;
        for (int p : sub) {
            const size_t bytes = (size_t)probs[p].first * probs[p].first * 8;
            CK(cudaMemcpyAsync(b2 + at, db + off[p], bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(c2 + at, dc + off[p], bytes, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(d2 + at, dd + off[p], bytes, cudaMemcpyDeviceToDevice, s));
            at += (int64_t)probs[p].first * probs[p].first;
        }
        sb = b2;
        sc = c2;
        sd = d2;
    }
    std::shared_ptr<DevPlan> dp;
    if ((rc = get_plan(keys, dp))) return rc;
    const bool plain = tol == 0.0 && !o.keep_levels && !o.timing;
    const TuneKey tk = tune_key(dp, o);
    Tune tu;
    if (!find_tune(tk, tu) && o.autotune && plain) {
        if ((rc = autotune(o, dp, keys, sb, sc, sd, tu))) return rc;
        store_tune(tk, tu);
    }
    tune_override(tu);
    if (o.graph && plain) {
        std::shared_ptr<GraphEntry> E = find_graph(tk, tu);
        if (E) return replay(*E, o, keys, sb, sc, sd, total, Hs, code, growth);
        // first build of this plan: as usual, while the sizes of its allocations are summed,
        // then recorded into a graph with buffers of its own for the later builds
        BumpCtx meas;
        meas.measure = true;
        for (const auto &k : keys) Hs.push_back(new_handle(k, o.precision));
        tl_bump = &meas;
        rc = run_build(o, tol, dp, sb, sc, sd, Hs, code, growth, tu);
        tl_bump = nullptr;
        if (rc == GM_OK) record_graph(o, tol, dp, keys, total, tu, tk, meas.total, Hs);
        return rc;
    }
    for (const auto &k : keys) Hs.push_back(new_handle(k, o.precision));
    return run_build(o, tol, dp, sb, sc, sd, Hs, code, growth, tu);
}

// Build with the automatic fallback; on failure every handle is freed.  In the mixed-
// precision default (block pivoting, GM_PIVOT_AUTO), problems whose reaction term makes
// the operator indefinite -- d below -2 pi^2 everywhere: the first Dirichlet eigenfunction
// of -Laplace on the unit square (eigenvalue 2 pi^2) then has a negative energy -- are
// built in FP64 from the start, and the problems whose mixed build raised the growth
// flag, refined too slowly or met a singular pivot are built again in FP64.
int build_with_fallback(const gm_opts &o, double tol, const std::vector<std::pair<int, int>> &probs,
                        const double *db, const double *dc, const double *dd, std::vector<gm_handle *> &H) {
    for (gm_handle *h : H) gm_free(h);
    H.assign(probs.size(), nullptr);
    std::vector<int64_t> off(probs.size() + 1, 0);
    for (size_t p = 0; p < probs.size(); ++p) off[p + 1] = off[p] + (int64_t)probs[p].first * probs[p].first;
    const bool autom = o.precision == GM_PREC_MIXED && o.pivoting == GM_PIVOT_AUTO;
    std::vector<int> mixed_set, fp64_set, all;
    for (size_t p = 0; p < probs.size(); ++p) all.push_back((int)p);
    int rc = GM_OK;
    auto finish = [&](int r) {
        if (r) {
            cudaGetLastError();
            for (gm_handle *&h : H) {
                gm_free(h);
                h = nullptr;
            }
            H.clear();
        }
        return r;
    };
    if (autom) {
        std::vector<double> maxd;
        if ((rc = max_reaction(probs, dd, (cudaStream_t)o.stream, maxd))) return finish(rc);
        const double lam1 = 2.0 * 3.14159265358979323846 * 3.14159265358979323846;
        for (int p : all) (maxd[p] < -lam1 ? fp64_set : mixed_set).push_back(p);
    } else {
        mixed_set = all;  // "mixed" here means: as requested
    }
    if (!mixed_set.empty()) {
        std::vector<gm_handle *> Hs;
        std::vector<int> code, growth;
        rc = build_subset(o, tol, probs, off, mixed_set, db, dc, dd, Hs, code, growth);
        for (size_t q = 0; q < Hs.size(); ++q) H[mixed_set[q]] = Hs[q];
        if (rc && !(autom && rc == GM_ESINGULAR)) return finish(rc);
        rc = GM_OK;
        if (autom)
            for (size_t q = 0; q < mixed_set.size(); ++q)
                if (growth[q] || code[q] == GM_ESINGULAR) fp64_set.push_back(mixed_set[q]);
    }
    if (!fp64_set.empty()) {
        std::sort(fp64_set.begin(), fp64_set.end());
        gm_opts o2 = o;
        o2.precision = GM_PREC_FP64;
        o2.pivoting = GM_PIVOT_PARTIAL;
        o2.panel_width = 0;
        std::vector<gm_handle *> Hs;
        std::vector<int> code, growth;
        rc = build_subset(o2, tol, probs, off, fp64_set, db, dc, dd, Hs, code, growth);
        for (size_t q = 0; q < Hs.size(); ++q) {
            gm_free(H[fp64_set[q]]);
            H[fp64_set[q]] = Hs[q];
            Hs[q]->info.pivot_fallback = 1;
        }
        if (rc) return finish(rc);
    }
    return GM_OK;
}

int check_opts(const gm_opts *opts, gm_opts &o) {
    gm_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != GM_PREC_FP64 && o.precision != GM_PREC_MIXED) return GM_EINVAL;
    if (o.pivoting < GM_PIVOT_AUTO || o.pivoting > GM_PIVOT_PARTIAL) return GM_EINVAL;
    if (o.hbs_leaf == 0) o.hbs_leaf = 64;
    if (o.hbs_leaf < 2 || o.hbs_leaf > 192) return GM_EINVAL;
    if (o.hbs_min_edge == 0) o.hbs_min_edge = 128;
    if (o.hbs_min_edge < 4) return GM_EINVAL;
    return GM_OK;
}

}  // namespace

extern "C" {

void gm_debug_fail_alloc(long long n) { g_fail_countdown.store(n > 0 ? n : 0); }

void gm_opts_default(gm_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = GM_PREC_FP64;
}

const char *gm_strerror(int code) {
    switch (code) {
    case GM_OK: return "ok";
    case GM_EINVAL: return "invalid argument";
    case GM_ENOMEM: return "out of memory";
    case GM_ESINGULAR: return "singular pivot: a box's Dirichlet problem is singular";
    case GM_ETIMEOUT: return "device wait timed out";
    case GM_ECUDA: return "CUDA runtime error";
    case GM_EUNSUPPORTED: return "unsupported request";
    case GM_ESCRATCH: return "request exceeds the fixed 16 MiB scratch of gm_solve_static";
    default: return "unknown error";
    }
}

void gm_free(gm_handle *h) {
    if (!h) return;
    cudaFree(h->T);
    cudaFree(h->Tdf);
    cudaFree(h->tdig);
    cudaFree(h->tex);
    cudaFree(h->F);
    cudaFree(h->FL);
    cudaFree(h->FR);
    for (void *p : h->kept_bufs) cudaFree(p);
    if (h->hbs) {
        gm::hbs_free(*h->hbs);
        delete h->hbs;
    }
    delete h;
}

int gm_build(const double *b, const double *c, const double *d, int n, int leaf, double tol, gm_handle **out) {
    gm_opts o;
    gm_opts_default(&o);
    return gm_build_ex(&o, b, c, d, n, leaf, tol, out);
}

int gm_build_ex(const gm_opts *opts, const double *b, const double *c, const double *d, int n, int leaf, double tol,
                gm_handle **out) {
    if (!out) return GM_EINVAL;
    *out = nullptr;
    if (!b || !c || !d || n < 2 || leaf < 3 || !(tol >= 0.0)) return GM_EINVAL;
    gm_opts o;
    int rc = check_opts(opts, o);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)o.stream;
    // coefficients on the device (device pointers are used in place)
    DBuf coef;
    const double *db = b, *dc = c, *dd = d;
    const size_t N2 = (size_t)n * n;
    if (!is_device_ptr(b) || !is_device_ptr(c) || !is_device_ptr(d)) {
        if ((rc = coef.alloc(3 * N2 * sizeof(double), s))) return rc;
        double *base = coef.as<double>();
        CK(cudaMemcpyAsync(base, b, N2 * 8, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(base + N2, c, N2 * 8, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(base + 2 * N2, d, N2 * 8, cudaMemcpyDefault, s));
        db = base;
        dc = base + N2;
        dd = base + 2 * N2;
    }
    std::vector<gm_handle *> H;
    rc = build_with_fallback(o, tol, {{n, leaf}}, db, dc, dd, H);
    if (rc) return rc;
    *out = H[0];
    return GM_OK;
}

int gm_build_batch(int count, const gm_problem *probs, const gm_opts *opts, double tol, gm_handle **outs) {
    if (count <= 0 || !probs || !outs || !(tol >= 0.0)) return GM_EINVAL;
    for (int i = 0; i < count; ++i) outs[i] = nullptr;
    std::vector<std::pair<int, int>> key;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        const gm_problem &p = probs[i];
        if (!p.b || !p.c || !p.d || p.n < 2 || p.leaf < 3) return GM_EINVAL;
        key.push_back({p.n, p.leaf});
        total += (int64_t)p.n * p.n;
    }
    gm_opts o;
    int rc = check_opts(opts, o);
    if (rc) return rc;
    if (o.keep_levels) return GM_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)o.stream;
    // every problem's coefficients, concatenated in batch order
    DBuf coef;
    if ((rc = coef.alloc(3 * (size_t)total * sizeof(double), s))) return rc;
    double *db = coef.as<double>(), *dc = db + total, *dd = dc + total;
    int64_t off = 0;
    for (int i = 0; i < count; ++i) {
        const size_t bytes = (size_t)probs[i].n * probs[i].n * 8;
        CK(cudaMemcpyAsync(db + off, probs[i].b, bytes, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(dc + off, probs[i].c, bytes, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(dd + off, probs[i].d, bytes, cudaMemcpyDefault, s));
        off += (int64_t)probs[i].n * probs[i].n;
    }
    std::vector<gm_handle *> H;
    rc = build_with_fallback(o, tol, key, db, dc, dd, H);
    if (rc) return rc;
    for (int i = 0; i < count; ++i) outs[i] = H[i];
    return GM_OK;
}

int gm_solve(gm_handle *h, const double *g, double *dudn, int batch, void *stream) {
    if (!h || batch < 0) return GM_EINVAL;
    if (batch == 0) return GM_OK;
    if (!g || !dudn) return GM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = 4 * h->n;
    const size_t bytes = (size_t)N * batch * 8;
    bool gd = is_device_ptr(g), vd = is_device_ptr(dudn);
    if (gd && vd && overlaps(g, dudn, (size_t)N * batch)) return GM_EINVAL;  // the apply reads g while it writes dudn
    DBuf gbuf, vbuf;
    const double *dg = g;
    double *dv = dudn;
    int rc;
    if (!gd) {
        if ((rc = gbuf.alloc(bytes, s))) return rc;
        CK(cudaMemcpyAsync(gbuf.p, g, bytes, cudaMemcpyHostToDevice, s));
        dg = gbuf.as<double>();
    }
    if (!vd) {
        if ((rc = vbuf.alloc(bytes, s))) return rc;
        dv = vbuf.as<double>();
    }
    if (h->hbs) {
        if ((rc = hbs_apply_dtn(*h->hbs, dg, dv, batch, s))) return rc;
    } else if (h->precision == GM_PREC_MIXED) {
        DBuf gdig, gex;
        if ((rc = gdig.alloc((size_t)h->split * batch * mx_kpad(N) * 2, s))) return rc;
        if ((rc = gex.alloc((size_t)batch * sizeof(int), s))) return rc;
        CK(mx_apply(h->tdig, h->tex, dg, gdig.as<__nv_bfloat16>(), gex.as<int>(), dv, N, batch, h->split, s));
    } else {
        CK(launch_apply(h->T, dg, dv, N, batch, s));
    }
    if (!vd) {
        CK(cudaMemcpyAsync(dudn, dv, bytes, cudaMemcpyDeviceToHost, s));
        gbuf.release();
        vbuf.release();
        CK(cudaStreamSynchronize(s));
    }
    return GM_OK;
}

int gm_solve_many(int count, gm_handle *const *hs, const double *const *g, double *const *dudn, const int *batch,
                  void *stream) {
    if (count < 0 || (count > 0 && (!hs || !g || !dudn || !batch))) return GM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || batch[i] < 0) return GM_EINVAL;
        if (batch[i] == 0) continue;
        if (!g[i] || !dudn[i] || !is_device_ptr(g[i]) || !is_device_ptr(dudn[i])) return GM_EINVAL;
    }
    std::vector<ApplyDesc> f64;
    std::map<int, std::vector<MxApplyDesc>> mx;  // by digits per operand
    std::map<int, int64_t> mx_planes, mx_cols;
    int rc;
    for (int i = 0; i < count; ++i) {
        gm_handle *h = hs[i];
        const int B = batch[i], N = 4 * h->n;
        if (B == 0) continue;
        if (h->hbs) {  // Algorithm 2 per operator
            if ((rc = hbs_apply_dtn(*h->hbs, g[i], dudn[i], B, s))) return rc;
        } else if (h->precision == GM_PREC_MIXED) {
            const int kpad = mx_kpad(N);
            MxApplyDesc q{};
            q.tdig = h->tdig;
            q.tex = h->tex;
            q.G = g[i];
            q.V = dudn[i];
            q.gplane = (int64_t)B * kpad;
            q.N = N;
            q.B = B;
            q.kpad = kpad;
            mx[h->split].push_back(q);
            mx_planes[h->split] += q.gplane;
            mx_cols[h->split] += B;
        } else {
            f64.push_back(ApplyDesc{h->T, g[i], dudn[i], N, B, 0, 0});
        }
    }
    DBuf d1;
    if (!f64.empty()) {
        if ((rc = d1.alloc(f64.size() * sizeof(ApplyDesc), s))) return rc;
        CK(launch_apply_many(f64, d1.as<ApplyDesc>(), s));
    }
    for (auto &kv : mx) {
        const int split = kv.first;
        std::vector<MxApplyDesc> &v = kv.second;
        DBuf dd, dig, ex;
        if ((rc = dd.alloc(v.size() * sizeof(MxApplyDesc), s)) ||
            (rc = dig.alloc((size_t)split * mx_planes[split] * 2, s)) ||
            (rc = ex.alloc((size_t)mx_cols[split] * sizeof(int), s)))
            return rc;
        int64_t po = 0, eo = 0;
        for (MxApplyDesc &q : v) {  // each operator's planes: split consecutive planes of gplane elements
            q.gdig = dig.as<__nv_bfloat16>() + po;
            q.gex = ex.as<int>() + eo;
            po += (int64_t)split * q.gplane;
            eo += q.B;
        }
        CK(mx_apply_many(v, dd.as<MxApplyDesc>(), split, s));
    }
    return GM_OK;
}

int gm_get_dtn(gm_handle *h, double *T_out) {
    if (!h || !T_out) return GM_EINVAL;
    if (h->hbs) return hbs_dense_dtn(*h->hbs, T_out, nullptr);
    size_t bytes = (size_t)16 * h->n * h->n * 8;
    CK(cudaMemcpy(T_out, h->T, bytes, cudaMemcpyDefault));
    return GM_OK;
}

int gm_get_schur(gm_handle *h, int x0, int y0, int a, int b, double *S_out) {
    if (!h || !S_out) return GM_EINVAL;
    if (h->kept.empty()) return GM_EUNSUPPORTED;
    for (auto &kv : h->kept) {
        const Box &bx = kv.first;
        if (bx.x0 == x0 && bx.y0 == y0 && bx.a == a && bx.b == b) {
            size_t r = (size_t)ring_size(a, b);
            if (!h->kept_df32) {
                CK(cudaMemcpy(S_out, kv.second, r * r * 8, cudaMemcpyDefault));
                return GM_OK;
            }
            std::vector<float2> tmp(r * r);
            std::vector<double> out(r * r);
            CK(cudaMemcpy(tmp.data(), kv.second, r * r * sizeof(float2), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < r * r; ++i) out[i] = (double)tmp[i].x + (double)tmp[i].y;
            CK(cudaMemcpy(S_out, out.data(), r * r * 8, cudaMemcpyDefault));
            return GM_OK;
        }
    }
    return GM_EINVAL;
}

int gm_info(gm_handle *h, gm_info_t *info) {
    if (!h || !info) return GM_EINVAL;
    *info = h->info;
    return GM_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- body loads

namespace {

// The FP64 build with body loads (Section 6.3) of one problem: the plain build's leaves,
// merges and root, each merge's interface system widened by its children's load columns,
// the leaves' load maps from their own [A_ii | E_i] systems, and the root's load columns
// beside [S_root | B].  Gives h->T and h->F.
int run_build_loads(const gm_opts &o, int n, int leaf, const std::vector<int> &body, const double *db,
                    const double *dc, const double *dd, gm_handle *h) {
    cudaStream_t s = (cudaStream_t)o.stream;
    int rc;
    std::shared_ptr<DevPlan> dpp;
    if ((rc = get_plan({{n, leaf}}, dpp))) return rc;
    const DevPlan &dp = *dpp;
    const Plan &P = dp.plan;
    if (leaf_smem_bytes(dp.max_leaf_a, dp.max_leaf_b) > 220 * 1024) return GM_EUNSUPPORTED;
    if (2 * (dp.max_leaf_a - 2) + 2 * (dp.max_leaf_b - 2) - 4 > 64) return GM_EUNSUPPORTED;
    const int nb = o.panel_width > 0 ? o.panel_width : 16;
    if (nb > GJ_MAX_NB) return GM_EINVAL;
    LoadPlan lp;
    if ((rc = build_load_plan(P, body, lp))) return rc;
    h->plan = dpp;
    h->L = P.L;
    const RootDesc &R = P.roots[0];
    const int r = R.r, nb4 = 4 * n, m = lp.nbody;
    KTimer kt;

    auto put = [&](DBuf &buf, const void *src, size_t bytes) -> int {
        int e = buf.alloc(bytes, s);
        if (e) return e;
        if (bytes) CK(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
        return GM_OK;
    };
    DBuf stat;
    Status hst{0, -1, 0x7ff0000000000000ull, 0, 0u};
    if ((rc = put(stat, &hst, sizeof(Status)))) return rc;
    Status *dst = stat.as<Status>();
    DBuf arena, larena;
    if ((rc = arena.alloc((size_t)P.arena_doubles * 8, s)) || (rc = larena.alloc((size_t)lp.arena * 8, s))) return rc;
    double *A64 = arena.as<double>(), *LA = larena.as<double>();

    // scratch of the dense sweeps: the leaves' systems, every stage, the root
    const SysDesc root_sys{0, r, r + nb4 + m, 0, 0, 0, 0};
    int max_nm = std::max<int>(1, (int)lp.leaf_sys.size()), piv_ld = std::max(r, lp.leaf_max_m);
    int64_t max_u12 = std::max<int64_t>((int64_t)lp.leaf_sys.size() * nb * lp.leaf_max_ncol,
                                        (int64_t)nb * root_sys.ncol);
    for (size_t si = 0; si < dp.stages.size(); ++si) {
        max_nm = std::max(max_nm, dp.stages[si].nm);
        piv_ld = std::max(piv_ld, dp.stages[si].max_m);
        max_u12 = std::max<int64_t>(max_u12, (int64_t)dp.stages[si].nm * nb * lp.stage_max_ncol[si]);
    }
    DBuf piv, u12;
    if ((rc = piv.alloc((size_t)max_nm * piv_ld * sizeof(int), s)) || (rc = u12.alloc((size_t)max_u12 * 8, s)))
        return rc;

    // leaves: Schur complements, then the load maps of the leaves that hold body nodes
    CK(launch_leaf(dp.d_leaves, P.leaves, dp.max_leaf_a, dp.max_leaf_b, db, dc, dd, A64, dst, 0, s, kt));
    DBuf d_leaves, d_nodes, d_lsys, lws;
    const int nl = (int)lp.leaves.size();
    if ((rc = put(d_leaves, lp.leaves.data(), lp.leaves.size() * sizeof(LeafLoadDesc))) ||
        (rc = put(d_nodes, lp.leaf_nodes.data(), lp.leaf_nodes.size() * sizeof(int))) ||
        (rc = put(d_lsys, lp.leaf_sys.data(), lp.leaf_sys.size() * sizeof(SysDesc))) ||
        (rc = lws.alloc((size_t)lp.leaf_ws * 8, s)))
        return rc;
    int64_t max_le = 0, max_rm = 0;
    for (const LeafLoadDesc &d : lp.leaves) {
        max_le = std::max<int64_t>(max_le, (int64_t)d.ni * (d.ni + d.m));
        max_rm = std::max<int64_t>(max_rm, (int64_t)ring_size(d.a, d.b) * d.m);
    }
    if (!lp.leaf_sys.empty()) {
        CK(launch_leaf_load_assemble(d_leaves.as<LeafLoadDesc>(), nl, d_nodes.as<int>(), lws.as<double>(),
                                     (int)max_le, db, dc, dd, s));
        CK(launch_gj_sweep(d_lsys.as<SysDesc>(), lp.leaf_sys, lp.leaf_max_m, lp.leaf_max_ncol, lws.as<double>(), nb,
                           piv.as<int>(), piv_ld, u12.as<double>(), (int64_t)nb * lp.leaf_max_ncol, dst, 0, s, kt));
    }
    CK(launch_leaf_load_finalize(d_leaves.as<LeafLoadDesc>(), nl, d_nodes.as<int>(), lws.as<double>(), LA,
                                 (int)max_rm, db, dc, dd, s));

    // merge stages: [M | Z | Z_L] swept together; S and the load map of every parent
    for (size_t si = 0; si < dp.stages.size(); ++si) {
        const DevStage &ds = dp.stages[si];
        if (ds.nm == 0) continue;
        const std::vector<MergeDesc> &mc = lp.merges[si];
        DBuf d_mc, d_ml, d_sys, ws;
        if ((rc = put(d_mc, mc.data(), mc.size() * sizeof(MergeDesc))) ||
            (rc = put(d_ml, lp.stages[si].data(), lp.stages[si].size() * sizeof(MergeLoadDesc))) ||
            (rc = put(d_sys, lp.sys[si].data(), lp.sys[si].size() * sizeof(SysDesc))) ||
            (rc = ws.alloc((size_t)lp.stage_ws[si] * 8, s)))
            return rc;
        int64_t max_e = 0, max_l = 0;
        for (size_t k = 0; k < mc.size(); ++k) {
            const int64_t mm = 2 * mc[k].sp, mL = lp.stages[si][k].m1 + lp.stages[si][k].m2;
            max_e = std::max(max_e, mm * (mm + mc[k].rp));
            max_l = std::max(max_l, std::max(mm, (int64_t)mc[k].rp) * mL);
        }
        CK(launch_merge_assemble(d_mc.as<MergeDesc>(), ds.nm, ds.d_tab, A64, ws.as<double>(), max_e, db, dc, dd, 0,
                                 s, kt));
        CK(launch_merge_load_assemble(d_mc.as<MergeDesc>(), d_ml.as<MergeLoadDesc>(), ds.nm, ds.d_tab, LA,
                                      ws.as<double>(), max_l, s));
        CK(launch_gj_sweep(d_sys.as<SysDesc>(), lp.sys[si], ds.max_m, lp.stage_max_ncol[si], ws.as<double>(), nb,
                           piv.as<int>(), piv_ld, u12.as<double>(), (int64_t)nb * lp.stage_max_ncol[si], dst,
                           (int)si + 1, s, kt));
        CK(launch_merge_update(d_mc.as<MergeDesc>(), mc, ds.d_tab, A64, ws.as<double>(), A64, ds.max_rp, db, dc, dd,
                               0, s, kt));
        CK(launch_merge_load_update(d_mc.as<MergeDesc>(), d_ml.as<MergeLoadDesc>(), ds.nm, ds.d_tab, A64,
                                    ws.as<double>(), LA, max_l, s));
    }

    // root: [S_root | B | L_root] -> [* | S^{-1} B | S^{-1} L_root], then T and F
    DBuf rws, d_rsys, d_order;
    const std::vector<SysDesc> rsys{root_sys};
    if ((rc = rws.alloc((size_t)r * root_sys.ncol * 8, s)) || (rc = put(d_rsys, rsys.data(), sizeof(SysDesc))) ||
        (rc = put(d_order, lp.root_order.data(), lp.root_order.size() * sizeof(int))))
        return rc;
    double *W = rws.as<double>();
    CK(launch_root_assemble(A64 + R.off, r, n, W, db, dc, dd, s, kt));
    CK(cudaMemcpyAsync(W + (int64_t)r * (r + nb4), LA + lp.root_l, (size_t)r * m * 8, cudaMemcpyDeviceToDevice, s));
    CK(launch_gj_sweep(d_rsys.as<SysDesc>(), rsys, r, root_sys.ncol, W, nb, piv.as<int>(), piv_ld, u12.as<double>(),
                       (int64_t)nb * root_sys.ncol, dst, (int)dp.stages.size() + 1, s, kt));
    cudaError_t e = cudaMalloc(&h->T, (size_t)nb4 * nb4 * 8);
    if (e == cudaSuccess) e = cudaMalloc(&h->F, (size_t)nb4 * m * 8);
    if (e != cudaSuccess) return alloc_error(e);
    CK(launch_root_finalize(W, r, n, h->T, s, kt));
    CK(launch_load_finalize(W + (int64_t)r * (r + nb4), r, n, m, d_order.as<int>(), h->F, s));
    h->nbody = m;

    CK(cudaMemcpyAsync(&hst, stat.p, sizeof(Status), cudaMemcpyDeviceToHost, s));
    for (DBuf *b : {&rws, &d_rsys, &d_order, &lws, &d_leaves, &d_nodes, &d_lsys, &piv, &u12, &arena, &larena, &stat})
        b->release();
    CK(cudaStreamSynchronize(s));
    gm_info_t info{};
    for (int f = 0; f < GM_K_NFAM; ++f) {
        info.kernel_launches[f] = kt.launches[f];
        info.kernel_flops[f] = kt.flops[f];
        info.launches += kt.launches[f];
    }
    double mp;
    memcpy(&mp, &hst.min_piv, 8);
    info.n = n;
    info.leaf = leaf;
    info.levels = P.L_user;
    info.load_rank = -1;
    info.precision = GM_PREC_FP64;
    info.pivoting = GM_PIVOT_PARTIAL;
    info.dtn_bytes = (long long)nb4 * nb4 * 8;
    info.resident_bytes = info.dtn_bytes + (long long)nb4 * m * 8;
    info.peak_workspace = (int64_t)(P.arena_doubles + lp.arena + (int64_t)r * root_sys.ncol) * 8;
    info.min_pivot_ratio = mp / (4.0 * (n + 1.0) * (n + 1.0));
    info.bad_stage = hst.code ? hst.where : -1;
    h->info = info;
    return hst.code;
}

}  // namespace

extern "C" {

int gm_build_loads(const gm_opts *opts, const double *b, const double *c, const double *d, int n, int leaf,
                   const int *body, int nbody, gm_handle **out) {
    if (!out) return GM_EINVAL;
    *out = nullptr;
    if (!b || !c || !d || n < 2 || leaf < 3 || !body || nbody < 1 || (int64_t)nbody > (int64_t)n * n)
        return GM_EINVAL;
    gm_opts o;
    int rc = check_opts(opts, o);
    if (rc) return rc;
    if (o.precision != GM_PREC_FP64 || o.keep_levels) return GM_EUNSUPPORTED;
    const std::vector<int> nodes(body, body + nbody);
    const int64_t N2 = (int64_t)n * n;
    std::vector<int> sorted(nodes);
    std::sort(sorted.begin(), sorted.end());
    if (sorted.front() < 0 || sorted.back() >= N2 || std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return GM_EINVAL;
    cudaStream_t s = (cudaStream_t)o.stream;
    DBuf coef;
    const double *db = b, *dc = c, *dd = d;
    if (!is_device_ptr(b) || !is_device_ptr(c) || !is_device_ptr(d)) {
        if ((rc = coef.alloc(3 * (size_t)N2 * sizeof(double), s))) return rc;
        double *base = coef.as<double>();
        CK(cudaMemcpyAsync(base, b, N2 * 8, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(base + N2, c, N2 * 8, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(base + 2 * N2, d, N2 * 8, cudaMemcpyDefault, s));
        db = base;
        dc = base + N2;
        dd = base + 2 * N2;
    }
    gm_handle *h = new_handle({n, leaf}, GM_PREC_FP64);
    rc = run_build_loads(o, n, leaf, nodes, db, dc, dd, h);
    if (rc) {
        gm_free(h);
        return rc;
    }
    *out = h;
    return GM_OK;
}

int gm_solve_loads(gm_handle *h, const double *g, const double *f, double *dudn, int batch, void *stream) {
    if (!h || batch < 0) return GM_EINVAL;
    if (!h->F && h->frank < 0) return GM_EUNSUPPORTED;
    if (batch == 0) return GM_OK;
    if (!g || !f || !dudn) return GM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = 4 * h->n, m = h->nbody;
    const size_t gbytes = (size_t)N * batch * 8, fbytes = (size_t)m * batch * 8;
    DBuf gbuf, fbuf, vbuf;
    const double *dg = g, *df = f;
    double *dv = dudn;
    int rc;
    if (!is_device_ptr(g)) {
        if ((rc = gbuf.alloc(gbytes, s))) return rc;
        CK(cudaMemcpyAsync(gbuf.p, g, gbytes, cudaMemcpyHostToDevice, s));
        dg = gbuf.as<double>();
    }
    if (!is_device_ptr(f)) {
        if ((rc = fbuf.alloc(fbytes, s))) return rc;
        CK(cudaMemcpyAsync(fbuf.p, f, fbytes, cudaMemcpyHostToDevice, s));
        df = fbuf.as<double>();
    }
    const bool vd = is_device_ptr(dudn);
    if (!vd) {
        if ((rc = vbuf.alloc(gbytes, s))) return rc;
        dv = vbuf.as<double>();
    }
    CK(launch_apply(h->T, dg, dv, N, batch, s));
    if (h->frank < 0) {
        CK(launch_apply_add(h->F, df, dv, N, m, batch, s));
    } else if (h->frank > 0) {  // the low-rank form: dudn += FL (FR f)
        const int k = h->frank;
        DBuf w;
        if ((rc = w.alloc((size_t)k * batch * 8, s))) return rc;
        if ((rc = hbs_gemm(h->FR, k, 0, df, m, 0, w.as<double>(), k, k, batch, m, 1.0, 0.0, s)) ||
            (rc = hbs_gemm(h->FL, N, 0, w.as<double>(), k, 0, dv, N, N, batch, k, 1.0, 1.0, s)))
            return rc;
    }
    if (!vd) {
        CK(cudaMemcpyAsync(dudn, dv, gbytes, cudaMemcpyDeviceToHost, s));
        gbuf.release();
        fbuf.release();
        vbuf.release();
        CK(cudaStreamSynchronize(s));
    }
    return GM_OK;
}

int gm_get_load_operator(gm_handle *h, double *F_out) {
    if (!h || !F_out) return GM_EINVAL;
    const size_t N = 4 * (size_t)h->n, bytes = N * h->nbody * 8;
    if (h->frank >= 0) {  // the low-rank form, multiplied out
        DBuf t;
        int rc;
        if ((rc = t.alloc(bytes, nullptr))) return rc;
        CK(cudaMemsetAsync(t.p, 0, bytes, nullptr));
        if (h->frank > 0 && (rc = hbs_gemm(h->FL, (int)N, 0, h->FR, h->frank, 0, t.as<double>(), (int)N, (int)N,
                                           h->nbody, h->frank, 1.0, 0.0, nullptr)))
            return rc;
        CK(cudaMemcpyAsync(F_out, t.p, bytes, cudaMemcpyDefault, nullptr));
        CK(cudaStreamSynchronize(nullptr));
        return GM_OK;
    }
    if (!h->F) return GM_EUNSUPPORTED;
    CK(cudaMemcpy(F_out, h->F, bytes, cudaMemcpyDefault));
    return GM_OK;
}

int gm_compress_load_operator(gm_handle *h, double tol) {
    if (!h || !(tol > 0.0)) return GM_EINVAL;
    if (!h->F) return GM_EUNSUPPORTED;  // no loads, or already compressed
    const int N = 4 * h->n;
    double *L = nullptr, *R = nullptr;
    int k = 0;
    int rc = hbs_lowrank(h->F, N, h->nbody, tol, nullptr, &L, &R, &k);
    if (rc) return rc;
    cudaFree(h->F);
    h->F = nullptr;
    h->FL = L;
    h->FR = R;
    h->frank = k;
    h->info.load_rank = k;
    h->info.resident_bytes = (long long)N * N * 8 + (long long)(N + h->nbody) * k * 8;
    return GM_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- networks

extern "C" {

int gm_build_net(const gm_opts *opts, const double *sx, const double *sy, int n, int leaf, double tol,
                 const int *body, int nbody, gm_handle **out) {
    if (!out) return GM_EINVAL;
    *out = nullptr;
    if (!sx || !sy || n < 2 || leaf < 3 || !(tol >= 0.0) || nbody < 0 || (nbody > 0 && !body) ||
        (int64_t)nbody > (int64_t)n * n)
        return GM_EINVAL;
    gm_opts o;
    int rc = check_opts(opts, o);
    if (rc) return rc;
    if (o.precision != GM_PREC_FP64 || (nbody > 0 && (o.keep_levels || tol > 0.0))) return GM_EUNSUPPORTED;
    std::vector<int> nodes(body, body + nbody);
    if (nbody > 0) {
        std::vector<int> sorted(nodes);
        std::sort(sorted.begin(), sorted.end());
        if (sorted.front() < 0 || sorted.back() >= (int64_t)n * n ||
            std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return GM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)o.stream;
    const size_t L = (size_t)n * (n + 1);
    DBuf links, wts, sig;
    const double *dsx = sx, *dsy = sy;
    if (!is_device_ptr(sx) || !is_device_ptr(sy)) {
        if ((rc = links.alloc(2 * L * sizeof(double), s))) return rc;
        CK(cudaMemcpyAsync(links.p, sx, L * 8, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(links.as<double>() + L, sy, L * 8, cudaMemcpyDefault, s));
        dsx = links.as<double>();
        dsy = dsx + L;
    }
    if ((rc = wts.alloc((size_t)5 * n * n * sizeof(double), s)) || (rc = sig.alloc((size_t)4 * n * sizeof(double), s)))
        return rc;
    CK(launch_net_weights(dsx, dsy, n, wts.as<double>(), sig.as<double>(), s));
    // the FP64 build on the weight table (a null c pointer selects it)
    const double *W = wts.as<double>();
    gm_handle *h = nullptr;
    if (nbody == 0) {
        std::vector<gm_handle *> H;
        if ((rc = build_with_fallback(o, tol, {{n, leaf}}, W, nullptr, W, H))) return rc;
        h = H[0];
    } else {
        h = new_handle({n, leaf}, GM_PREC_FP64);
        if ((rc = run_build_loads(o, n, leaf, nodes, W, nullptr, W, h))) {
            gm_free(h);
            return rc;
        }
    }
    // the datum at ghost k is the current through its link: rows of T and F times sigma_k
    // (an HBS root keeps the conductivities and weights every apply instead)
    cudaError_t e = cudaSuccess;
    if (h->hbs) {
        e = cudaMalloc(&h->hbs->sig, (size_t)4 * n * sizeof(double));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->hbs->sig, sig.p, (size_t)4 * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
        e = launch_scale_rows(h->T, 4 * n, 4 * n, sig.as<double>(), s);
    }
    if (e == cudaSuccess && h->F) e = launch_scale_rows(h->F, 4 * n, nbody, sig.as<double>(), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        gm_free(h);
        return cuda_fail(e, "network datum weights", __LINE__);
    }
    *out = h;
    return GM_OK;
}

}  // extern "C"
