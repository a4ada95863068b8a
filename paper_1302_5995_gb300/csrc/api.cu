// C ABI: gm_build / gm_solve / gm_get_dtn / gm_get_schur / gm_info / gm_free.
//
// The build runs the paper's level-by-level sweep (Section 3.3): every leaf in one
// launch, then per level one stage of horizontal pairwise merges and one of vertical
// ones (each stage batched over all its merges), then the root.  All device memory is
// taken from the CUDA stream-ordered allocator on the build stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "gm_internal.h"
#include "kernels.h"
#include "mixed.h"
#include "blocked.h"

using namespace gm;

namespace {

#define CK(x)                                       \
    do {                                            \
        cudaError_t _e = (x);                       \
        if (_e != cudaSuccess) return GM_ECUDA;     \
    } while (0)

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device buffer released on scope exit through the stream-ordered allocator.
struct DBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
    int alloc(size_t bytes, cudaStream_t st) {
        release();
        s = st;
        if (bytes == 0) bytes = 16;
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return GM_ENOMEM;
        }
        return GM_OK;
    }
    template <class T> T *as() const { return (T *)p; }
};

// Device copy of a plan (cached per (n, leaf) and per device).
struct DevStage {
    int orient, nm, max_m, max_ncol, max_rp;
    int sum_rows = 0, sum_cols = 0;
    int64_t in_doubles, out_doubles, ws_doubles, max_elems;
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

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int>, std::shared_ptr<DevPlan>> g_plans;

template <class T> int upload(T **dst, const std::vector<T> &v) {
    size_t bytes = v.size() * sizeof(T);
    if (cudaMalloc((void **)dst, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    if (bytes && cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) return GM_ECUDA;
    return GM_OK;
}

int get_plan(int n, int leaf, std::shared_ptr<DevPlan> &out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto key = std::make_tuple(dev, n, leaf);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        out = it->second;
        return GM_OK;
    }
    auto dp = std::make_shared<DevPlan>();
    int rc = build_plan(n, leaf, dp->plan);
    if (rc) return rc;
    for (const Box &b : dp->plan.leaf_boxes) {
        dp->max_leaf_a = std::max(dp->max_leaf_a, b.a);
        dp->max_leaf_b = std::max(dp->max_leaf_b, b.b);
    }
    if ((rc = upload(&dp->d_leaves, dp->plan.leaves))) return rc;
    for (const Stage &st : dp->plan.stages) {
        DevStage ds;
        ds.orient = st.orient;
        ds.nm = (int)st.merges.size();
        ds.max_m = st.max_m;
        ds.max_ncol = st.max_ncol;
        ds.max_rp = st.max_rp;
        ds.in_doubles = st.in_doubles;
        ds.out_doubles = st.out_doubles;
        ds.ws_doubles = st.ws_doubles;
        ds.max_elems = 0;
        std::vector<SysDesc> sys;
        int roff = 0, coff = 0;
        for (int i = 0; i < ds.nm; ++i) {
            const MergeDesc &m = st.merges[i];
            SysDesc s{m.ws, 2 * m.sp, 2 * m.sp + m.rp, i, roff, coff, 0};
            roff += s.m;
            coff += s.ncol;
            sys.push_back(s);
            ds.max_elems = std::max(ds.max_elems, (int64_t)s.m * s.ncol);
        }
        ds.sum_rows = roff;
        ds.sum_cols = coff;
        ds.h_sys = sys;
        dp->stages.push_back(ds);
        DevStage &d = dp->stages.back();
        if ((rc = upload(&d.d_merges, st.merges))) return rc;
        if ((rc = upload(&d.d_tab, st.table))) return rc;
        if ((rc = upload(&d.d_sys, sys))) return rc;
    }
    int r = dp->plan.r_root;
    std::vector<SysDesc> rs{SysDesc{0, r, r + 4 * n, 0, 0, 0, 0}};
    dp->h_root_sys = rs;
    if ((rc = upload(&dp->d_root_sys, rs))) return rc;
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
}  // namespace gm

struct gm_handle {
    int n = 0, leaf = 0, L = 0, precision = 0;
    double *T = nullptr;      // 4n x 4n column-major
    float2 *Tdf = nullptr;          // mixed precision: T as double-float
    __nv_bfloat16 *tdig = nullptr;  // mixed precision: digit planes of T's rows, for the apply
    int *tex = nullptr;             // mixed precision: row exponents of T
    int split = 4;            // mixed precision: digits per operand
    std::shared_ptr<DevPlan> plan;
    // kept intermediates: box -> device pointer of its Schur complement (FP64, or
    // double-float pairs for a mixed-precision build)
    std::vector<std::pair<Box, void *>> kept;
    bool kept_df32 = false;
    std::vector<void *> kept_bufs;
    gm_info_t info{};
};

const double *gm::handle_dtn(gm_handle *h, int *n) {
    if (!h) return nullptr;
    *n = h->n;
    return h->T;
}

extern "C" {

void gm_opts_default(gm_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = GM_PREC_FP64;
    o->panel_width = 8;
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
    for (void *p : h->kept_bufs) cudaFree(p);
    delete h;
}

int gm_build(const double *b, const double *c, const double *d, int n, int leaf, double tol, gm_handle **out) {
    gm_opts o;
    gm_opts_default(&o);
    return gm_build_ex(&o, b, c, d, n, leaf, tol, out);
}

static int build_impl(const gm_opts &o, const double *b, const double *c, const double *d, int n, int leaf,
                      gm_handle *H) {
    cudaStream_t s = (cudaStream_t)o.stream;
    int nb = o.panel_width > 0 ? o.panel_width : 8;
    if (nb > GJ_MAX_NB) return GM_EINVAL;
    std::shared_ptr<DevPlan> dp;
    int rc = get_plan(n, leaf, dp);
    if (rc) return rc;
    const Plan &P = dp->plan;
    if (leaf_smem_bytes(dp->max_leaf_a, dp->max_leaf_b) > 220 * 1024) return GM_EUNSUPPORTED;
    H->plan = dp;
    H->L = P.L;
    const size_t N2 = (size_t)n * n;
    // coefficients on the device
    DBuf coef;
    const double *db = b, *dc = c, *dd = d;
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
    DBuf stat;
    if ((rc = stat.alloc(sizeof(Status), s))) return rc;
    Status st0{0, -1, 0x7ff0000000000000ull, 0, 0};
    CK(cudaMemcpyAsync(stat.p, &st0, sizeof(st0), cudaMemcpyHostToDevice, s));
    Status *dst = stat.as<Status>();
    int64_t peak = 0;
    KTimer kt;
    kt.on = o.timing != 0;
    // A level's Schur complements: stream-ordered scratch, or handle-owned when kept.
    auto alloc_level = [&](size_t bytes, DBuf &owner, double *&ptr) -> int {
        if (o.keep_levels) {
            void *p = nullptr;
            if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
                cudaGetLastError();
                return GM_ENOMEM;
            }
            H->kept_bufs.push_back(p);
            ptr = (double *)p;
            return GM_OK;
        }
        int e = owner.alloc(bytes, s);
        ptr = owner.as<double>();
        return e;
    };
    auto keep = [&](const std::vector<Box> &boxes, const std::vector<int64_t> &offs, double *base) {
        if (!o.keep_levels) return;
        for (size_t i = 0; i < boxes.size(); ++i) H->kept.push_back({boxes[i], base + offs[i]});
    };

    // leaves (Section 3.3 step 2)
    DBuf cur_buf;
    double *cur_ptr = nullptr;
    if ((rc = alloc_level(P.leaf_doubles * 8, cur_buf, cur_ptr))) return rc;
    CK(launch_leaf(dp->d_leaves, P.leaves, dp->max_leaf_a, dp->max_leaf_b, db, dc, dd, n, cur_ptr, dst, 0, s,
                   kt));
    {
        std::vector<int64_t> offs;
        for (auto &l : P.leaves) offs.push_back(l.off);
        keep(P.leaf_boxes, offs, cur_ptr);
    }
    // merge stages (Section 3.3 step 3): per level, horizontal then vertical
    int piv_ld = P.r_root;
    int64_t max_u12 = (int64_t)nb * (P.r_root + 4 * n);
    int max_nm = 1;
    for (const DevStage &ds : dp->stages) {
        piv_ld = std::max(piv_ld, ds.max_m);
        max_u12 = std::max(max_u12, (int64_t)ds.nm * nb * ds.max_ncol);
        max_nm = std::max(max_nm, ds.nm);
    }
    DBuf piv, u12;
    if ((rc = piv.alloc((size_t)max_nm * piv_ld * sizeof(int), s))) return rc;
    if ((rc = u12.alloc((size_t)max_u12 * 8, s))) return rc;
    for (size_t si = 0; si < dp->stages.size(); ++si) {
        const DevStage &ds = dp->stages[si];
        const Stage &hs = P.stages[si];
        DBuf nxt_buf, ws;
        double *nxt_ptr = nullptr;
        if ((rc = alloc_level(ds.out_doubles * 8, nxt_buf, nxt_ptr))) return rc;
        if ((rc = ws.alloc(ds.ws_doubles * 8, s))) return rc;
        peak = std::max(peak, (int64_t)(ds.ws_doubles + ds.out_doubles + ds.in_doubles) * 8);
        CK(launch_merge_assemble(ds.d_merges, ds.nm, ds.d_tab, cur_ptr, ws.as<double>(), ds.max_elems, db, dc,
                                 dd, n, s, kt));
        CK(launch_gj_sweep(ds.d_sys, ds.h_sys, ds.max_m, ds.max_ncol, ws.as<double>(), nb, piv.as<int>(), piv_ld,
                           u12.as<double>(), (int64_t)nb * ds.max_ncol, dst, (int)si + 1, s, kt));
        CK(launch_merge_update(ds.d_merges, hs.merges, ds.d_tab, cur_ptr, ws.as<double>(), nxt_ptr, ds.max_rp, db,
                               dc, dd, n, s, kt));
        std::vector<int64_t> offs;
        for (auto &m : hs.merges) offs.push_back(m.out);
        keep(hs.out_boxes, offs, nxt_ptr);
        // stream-ordered: the previous level is freed after this stage's kernels
        cur_buf.release();
        std::swap(cur_buf.p, nxt_buf.p);
        std::swap(cur_buf.s, nxt_buf.s);
        cur_ptr = nxt_ptr;
    }
    // root (Section 3.3 step 4): X = S_root^{-1} B, then T = (I - P X)/h
    const int r = P.r_root, nb4 = 4 * n;
    DBuf rws;
    if ((rc = rws.alloc((size_t)r * (r + nb4) * 8, s))) return rc;
    peak = std::max(peak, (int64_t)r * (r + nb4) * 8);
    CK(launch_root_assemble(cur_ptr, r, n, rws.as<double>(), db, dc, dd, s, kt));
    CK(launch_gj_sweep(dp->d_root_sys, dp->h_root_sys, r, r + nb4, rws.as<double>(), nb, piv.as<int>(), piv_ld,
                       u12.as<double>(), (int64_t)nb * (r + nb4), dst, (int)dp->stages.size() + 1, s, kt));
    if (cudaMalloc(&H->T, (size_t)nb4 * nb4 * 8) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    CK(launch_root_finalize(rws.as<double>(), r, n, H->T, s, kt));
    Status st;
    CK(cudaMemcpyAsync(&st, stat.p, sizeof(st), cudaMemcpyDeviceToHost, s));
    // release temporaries (stream-ordered) before the final synchronisation
    rws.release();
    piv.release();
    u12.release();
    cur_buf.release();
    coef.release();
    stat.release();
    CK(cudaStreamSynchronize(s));
    double ih = 4.0 * (n + 1.0) * (n + 1.0);
    double mp;
    memcpy(&mp, &st.min_piv, 8);
    H->info.min_pivot_ratio = mp / ih;
    H->info.bad_stage = st.code ? st.where : -1;
    int launches = 0;
    for (int f = 0; f < GM_K_NFAM; ++f) {
        launches += kt.launches[f];
        H->info.kernel_launches[f] = kt.launches[f];
        H->info.kernel_flops[f] = kt.flops[f];
    }
    kt.collect(H->info.kernel_ms);
    H->info.launches = launches;
    H->info.peak_workspace = peak;
    if (st.code) return st.code;
    return GM_OK;
}

// Mixed precision (GM_PREC_MIXED): leaves in FP64, converted once to double-float;
// every stage and the root on double-float data with split-product tensor-core updates.
static int build_impl_mixed(const gm_opts &o, const double *b, const double *c, const double *d, int n, int leaf,
                            gm_handle *H, int *growth_out) {
    const bool blockpiv = o.pivoting != GM_PIVOT_PARTIAL;
    cudaStream_t s = (cudaStream_t)o.stream;
    int nb = o.panel_width > 0 ? o.panel_width : 16;
    if (nb > GJ_MAX_NB) return GM_EINVAL;
    int split = o.split_digits ? o.split_digits : 5;
    if (split < 3 || split > 6) return GM_EINVAL;
    H->split = split;
    std::shared_ptr<DevPlan> dp;
    int rc = get_plan(n, leaf, dp);
    if (rc) return rc;
    const Plan &P = dp->plan;
    if (leaf_smem_bytes(dp->max_leaf_a, dp->max_leaf_b) > 220 * 1024) return GM_EUNSUPPORTED;
    if (!blockpiv && (size_t)(P.r_root) * nb * sizeof(float) > 200 * 1024) return GM_EUNSUPPORTED;
    H->plan = dp;
    H->L = P.L;
    H->kept_df32 = true;
    const size_t N2 = (size_t)n * n;
    DBuf coef;
    const double *db = b, *dc = c, *dd = d;
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
    DBuf stat;
    if ((rc = stat.alloc(sizeof(Status), s))) return rc;
    Status st0{0, -1, 0x7ff0000000000000ull, 0, 0};
    CK(cudaMemcpyAsync(stat.p, &st0, sizeof(st0), cudaMemcpyHostToDevice, s));
    Status *dst = stat.as<Status>();
    int64_t peak = 0;
    KTimer kt;
    kt.on = o.timing != 0;
    auto alloc_level = [&](size_t elems, DBuf &owner, float2 *&ptr) -> int {
        size_t bytes = elems * sizeof(float2);
        if (o.keep_levels) {
            void *p = nullptr;
            if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
                cudaGetLastError();
                return GM_ENOMEM;
            }
            H->kept_bufs.push_back(p);
            ptr = (float2 *)p;
            return GM_OK;
        }
        int e = owner.alloc(bytes, s);
        ptr = owner.as<float2>();
        return e;
    };
    auto keep = [&](const std::vector<Box> &boxes, const std::vector<int64_t> &offs, float2 *base) {
        if (!o.keep_levels) return;
        for (size_t i = 0; i < boxes.size(); ++i) H->kept.push_back({boxes[i], (void *)(base + offs[i])});
    };
    // leaves (Section 3.3 step 2) in FP64, then one conversion to double-float
    DBuf leaf64, cur_buf;
    if ((rc = leaf64.alloc(P.leaf_doubles * 8, s))) return rc;
    CK(launch_leaf(dp->d_leaves, P.leaves, dp->max_leaf_a, dp->max_leaf_b, db, dc, dd, n, leaf64.as<double>(), dst,
                   0, s, kt));
    float2 *cur_ptr = nullptr;
    if ((rc = alloc_level(P.leaf_doubles, cur_buf, cur_ptr))) return rc;
    CK(mx_convert(leaf64.as<double>(), cur_ptr, P.leaf_doubles, s, kt));
    leaf64.release();
    {
        std::vector<int64_t> offs;
        for (auto &l : P.leaves) offs.push_back(l.off);
        keep(P.leaf_boxes, offs, cur_ptr);
    }
    // scratch of the sweeps (sized for the largest stage or the root) and of the Schur updates
    int max_nm = 1;
    int64_t max_rows = P.r_root, max_cols = P.r_root + 4 * n, max_plane = 16, max_exp = 1;
    for (size_t si = 0; si < dp->stages.size(); ++si) {
        const DevStage &ds = dp->stages[si];
        max_nm = std::max(max_nm, ds.nm);
        max_rows = std::max<int64_t>(max_rows, ds.sum_rows);
        max_cols = std::max<int64_t>(max_cols, ds.sum_cols);
        max_plane = std::max<int64_t>(max_plane, P.stages[si].dig_elems);
        max_exp = std::max<int64_t>(max_exp, P.stages[si].exp_elems);
    }
    DBuf perm, perm_n, a11, fdig, rdig, fex, rex, ydig, xdig, yex, xex;
    if ((rc = perm.alloc((size_t)max_nm * 4 * GJ_MAX_NB * sizeof(int), s))) return rc;
    if ((rc = perm_n.alloc((size_t)max_nm * sizeof(int), s))) return rc;
    if ((rc = a11.alloc((size_t)max_nm * GJ_MAX_NB * GJ_MAX_NB * sizeof(float2), s))) return rc;
    if ((rc = fdig.alloc((size_t)split * max_rows * 16 * 2, s))) return rc;
    if ((rc = rdig.alloc((size_t)split * max_cols * 16 * 2, s))) return rc;
    if ((rc = fex.alloc((size_t)max_rows * sizeof(int), s))) return rc;
    if ((rc = rex.alloc((size_t)max_cols * sizeof(int), s))) return rc;
    if ((rc = ydig.alloc((size_t)split * max_plane * 2, s))) return rc;
    if ((rc = xdig.alloc((size_t)split * max_plane * 2, s))) return rc;
    if ((rc = yex.alloc((size_t)max_exp * sizeof(int), s))) return rc;
    if ((rc = xex.alloc((size_t)max_exp * sizeof(int), s))) return rc;
    // block-pivoting scratch
    DBuf bxd, bad, bxe, bae, bpmag, bfdig, bfex, badig, br0d, bed, brdig, baex, br0e, bee, brex, br0;
    BlkScratch bscr;
    if (blockpiv) {
        const size_t sq = (size_t)max_nm * 64;
        if ((rc = bxd.alloc((size_t)split * sq * 64 * 2, s)) || (rc = bad.alloc((size_t)split * sq * 64 * 2, s)) ||
            (rc = bxe.alloc(sq * sizeof(int), s)) || (rc = bae.alloc(sq * sizeof(int), s)) ||
            (rc = bpmag.alloc(sq * sizeof(float), s)) ||
            (rc = bfdig.alloc((size_t)split * max_rows * 64 * 2, s)) ||
            (rc = bfex.alloc((size_t)max_rows * sizeof(int), s)) ||
            (rc = badig.alloc((size_t)split * max_cols * 64 * 2, s)) ||
            (rc = br0d.alloc((size_t)split * max_cols * 64 * 2, s)) ||
            (rc = bed.alloc((size_t)split * max_cols * 64 * 2, s)) ||
            (rc = brdig.alloc((size_t)split * max_cols * 64 * 2, s)) ||
            (rc = baex.alloc((size_t)max_cols * sizeof(int), s)) ||
            (rc = br0e.alloc((size_t)max_cols * sizeof(int), s)) ||
            (rc = bee.alloc((size_t)max_cols * sizeof(int), s)) ||
            (rc = brex.alloc((size_t)max_cols * sizeof(int), s)) ||
            (rc = br0.alloc((size_t)max_cols * 64 * sizeof(float2), s)))
            return rc;
        bscr.x_dig = bxd.as<__nv_bfloat16>();
        bscr.a11_dig = bad.as<__nv_bfloat16>();
        bscr.x_ex = bxe.as<int>();
        bscr.a11_ex = bae.as<int>();
        bscr.pmag = bpmag.as<float>();
        bscr.fdig = bfdig.as<__nv_bfloat16>();
        bscr.fex = bfex.as<int>();
        bscr.adig = badig.as<__nv_bfloat16>();
        bscr.r0dig = br0d.as<__nv_bfloat16>();
        bscr.edig = bed.as<__nv_bfloat16>();
        bscr.rdig = brdig.as<__nv_bfloat16>();
        bscr.aex = baex.as<int>();
        bscr.r0ex = br0e.as<int>();
        bscr.eex = bee.as<int>();
        bscr.rex = brex.as<int>();
        bscr.r0 = br0.as<float2>();
        bscr.growth = &dst->growth;
    }
    MxScratch scr;
    scr.perm = perm.as<int>();
    scr.perm_n = perm_n.as<int>();
    scr.a11inv = a11.as<float2>();
    scr.fdig = fdig.as<__nv_bfloat16>();
    scr.rdig = rdig.as<__nv_bfloat16>();
    scr.fex = fex.as<int>();
    scr.rex = rex.as<int>();
    for (size_t si = 0; si < dp->stages.size(); ++si) {
        const DevStage &ds = dp->stages[si];
        const Stage &hs = P.stages[si];
        if ((size_t)ds.max_m * nb * sizeof(float) > 200 * 1024) return GM_EUNSUPPORTED;
        DBuf nxt_buf, ws;
        float2 *nxt_ptr = nullptr;
        if ((rc = alloc_level(ds.out_doubles, nxt_buf, nxt_ptr))) return rc;
        if ((rc = ws.alloc(ds.ws_doubles * sizeof(float2), s))) return rc;
        peak = std::max(peak, (int64_t)(ds.ws_doubles + ds.out_doubles + ds.in_doubles) * 8);
        CK(mx_merge_assemble(ds.d_merges, ds.nm, ds.d_tab, cur_ptr, ws.as<float2>(), ds.max_elems, db, dc, dd, n, s,
                             kt));
        if (blockpiv) {
            bscr.inv_plane = (int64_t)ds.nm * 64 * 64;
            bscr.fplane = (int64_t)ds.sum_rows * 64;
            bscr.cplane = (int64_t)ds.sum_cols * 64;
            CK(blk_gj_sweep(ds.d_sys, ds.h_sys, ds.max_m, ds.max_ncol, ws.as<float2>(), split, bscr, dst, (int)si + 1,
                            s, kt));
        } else {
            scr.fplane = (int64_t)ds.sum_rows * 16;
            scr.rplane = (int64_t)ds.sum_cols * 16;
            CK(mx_gj_sweep(ds.d_sys, ds.h_sys, ds.max_m, ds.max_ncol, ws.as<float2>(), nb, split, scr, dst,
                           (int)si + 1, s, kt));
        }
        CK(mx_merge_update(ds.d_merges, hs.merges, ds.d_tab, cur_ptr, ws.as<float2>(), nxt_ptr, ds.max_rp, split,
                           ydig.as<__nv_bfloat16>(), yex.as<int>(), xdig.as<__nv_bfloat16>(), xex.as<int>(),
                           hs.dig_elems, db, dc, dd, n, s, kt));
        std::vector<int64_t> offs;
        for (auto &m : hs.merges) offs.push_back(m.out);
        keep(hs.out_boxes, offs, nxt_ptr);
        cur_buf.release();
        std::swap(cur_buf.p, nxt_buf.p);
        std::swap(cur_buf.s, nxt_buf.s);
        cur_ptr = nxt_ptr;
    }
    // root (Section 3.3 step 4)
    const int r = P.r_root, nb4 = 4 * n;
    DBuf rws;
    if ((rc = rws.alloc((size_t)r * (r + nb4) * sizeof(float2), s))) return rc;
    peak = std::max(peak, (int64_t)r * (r + nb4) * 8);
    CK(mx_root_assemble(cur_ptr, r, n, rws.as<float2>(), db, dc, dd, s, kt));
    if (blockpiv) {
        bscr.inv_plane = (int64_t)64 * 64;
        bscr.fplane = (int64_t)r * 64;
        bscr.cplane = (int64_t)(r + nb4) * 64;
        CK(blk_gj_sweep(dp->d_root_sys, dp->h_root_sys, r, r + nb4, rws.as<float2>(), split, bscr, dst,
                        (int)dp->stages.size() + 1, s, kt));
    } else {
        scr.fplane = (int64_t)r * 16;
        scr.rplane = (int64_t)(r + nb4) * 16;
        CK(mx_gj_sweep(dp->d_root_sys, dp->h_root_sys, r, r + nb4, rws.as<float2>(), nb, split, scr, dst,
                       (int)dp->stages.size() + 1, s, kt));
    }
    const int kpadT = mx_kpad(nb4);
    if (cudaMalloc(&H->T, (size_t)nb4 * nb4 * 8) != cudaSuccess ||
        cudaMalloc(&H->Tdf, (size_t)nb4 * nb4 * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&H->tdig, (size_t)split * nb4 * kpadT * 2) != cudaSuccess ||
        cudaMalloc(&H->tex, (size_t)nb4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    CK(mx_root_finalize(rws.as<float2>(), r, n, H->T, H->Tdf, H->tdig, H->tex, split, s, kt));
    Status st;
    CK(cudaMemcpyAsync(&st, stat.p, sizeof(st), cudaMemcpyDeviceToHost, s));
    rws.release();
    perm.release();
    perm_n.release();
    a11.release();
    fdig.release();
    rdig.release();
    fex.release();
    rex.release();
    ydig.release();
    xdig.release();
    yex.release();
    xex.release();
    for (DBuf *b : {&bxd, &bad, &bxe, &bae, &bpmag, &bfdig, &bfex, &badig, &br0d, &bed, &brdig, &baex, &br0e, &bee,
                    &brex, &br0})
        b->release();
    cur_buf.release();
    coef.release();
    stat.release();
    CK(cudaStreamSynchronize(s));
    double ih = 4.0 * (n + 1.0) * (n + 1.0);
    double mp;
    memcpy(&mp, &st.min_piv, 8);
    H->info.min_pivot_ratio = mp / ih;
    H->info.bad_stage = st.code ? st.where : -1;
    int launches = 0;
    for (int f = 0; f < GM_K_NFAM; ++f) {
        launches += kt.launches[f];
        H->info.kernel_launches[f] = kt.launches[f];
        H->info.kernel_flops[f] = kt.flops[f];
    }
    kt.collect(H->info.kernel_ms);
    H->info.launches = launches;
    H->info.peak_workspace = peak;
    H->info.pivoting = blockpiv ? GM_PIVOT_BLOCK : GM_PIVOT_PARTIAL;
    *growth_out = st.growth;
    if (st.code) return st.code;
    return GM_OK;
}

int gm_build_ex(const gm_opts *opts, const double *b, const double *c, const double *d, int n, int leaf, double tol,
                gm_handle **out) {
    if (!out) return GM_EINVAL;
    *out = nullptr;
    if (!b || !c || !d || n < 2 || leaf < 4 || tol < 0) return GM_EINVAL;
    if (tol != 0.0) return GM_EUNSUPPORTED;
    gm_opts o;
    gm_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision != GM_PREC_FP64 && o.precision != GM_PREC_MIXED) return GM_EINVAL;
    gm_handle *H = new gm_handle();
    H->n = n;
    H->leaf = leaf;
    H->precision = o.precision;
    int rc;
    if (o.precision == GM_PREC_MIXED) {
        if (o.pivoting < GM_PIVOT_AUTO || o.pivoting > GM_PIVOT_PARTIAL) {
            delete H;
            return GM_EINVAL;
        }
        int growth = 0;
        rc = build_impl_mixed(o, b, c, d, n, leaf, H, &growth);
        if (o.pivoting == GM_PIVOT_AUTO && (growth || rc == GM_ESINGULAR)) {
            // block pivoting was not safe for this operator: redo with partial pivoting
            gm_free(H);
            H = new gm_handle();
            H->n = n;
            H->leaf = leaf;
            H->precision = o.precision;
            gm_opts o2 = o;
            o2.pivoting = GM_PIVOT_PARTIAL;
            rc = build_impl_mixed(o2, b, c, d, n, leaf, H, &growth);
            H->info.pivot_fallback = 1;
        }
    } else {
        rc = build_impl(o, b, c, d, n, leaf, H);
        H->info.pivoting = GM_PIVOT_PARTIAL;
    }
    H->info.n = n;
    H->info.leaf = leaf;
    H->info.levels = H->L;
    H->info.precision = o.precision;
    H->info.dtn_bytes = (long long)16 * n * n * 8;
    if (rc) {
        cudaGetLastError();
        gm_free(H);
        return rc;
    }
    *out = H;
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
    DBuf gbuf, vbuf;
    const double *dg = g;
    double *dv = dudn;
    if (!gd) {
        if (gbuf.alloc(bytes, s)) return GM_ENOMEM;
        CK(cudaMemcpyAsync(gbuf.p, g, bytes, cudaMemcpyHostToDevice, s));
        dg = gbuf.as<double>();
    }
    if (!vd) {
        if (vbuf.alloc(bytes, s)) return GM_ENOMEM;
        dv = vbuf.as<double>();
    }
    if (h->precision == GM_PREC_MIXED) {
        DBuf gdig, gex;
        if (gdig.alloc((size_t)h->split * batch * mx_kpad(N) * 2, s)) return GM_ENOMEM;
        if (gex.alloc((size_t)batch * sizeof(int), s)) return GM_ENOMEM;
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

int gm_get_dtn(gm_handle *h, double *T_out) {
    if (!h || !T_out) return GM_EINVAL;
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
