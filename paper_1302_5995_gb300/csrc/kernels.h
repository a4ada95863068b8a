// Launchers of the CUDA kernels (host side).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "gm_internal.h"

#define LEAF_THREADS 256
#define GJ_PANEL_THREADS 512
#define GJ_MAX_NB 16

namespace gm {

// Stream-ordered device allocation from the library's memory pool (which keeps freed
// memory mapped for later calls); free with cudaFreeAsync on a stream.  GM_ENOMEM when
// the device is out of memory, GM_ECUDA for other failures.
int dev_alloc(void **p, size_t bytes, cudaStream_t s);

// Process-wide pool of timing events (created once, reused by every timed build).
cudaEvent_t event_pool_get();
void event_pool_put(cudaEvent_t e);

// Per-family launch accounting: algorithmic flops are always counted; with `on`, every
// launch is bracketed by a pair of pooled CUDA events on its stream.
struct KTimer {
    bool on = false;
    unsigned mask = ~0u;  // families whose launches are timed (bit f = family f)
    bool open = false;    // the last begin() recorded an event pair
    double flops[GM_K_NFAM] = {};
    int launches[GM_K_NFAM] = {};
    struct Rec {
        int fam;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    KTimer() = default;
    KTimer(const KTimer &) = delete;
    KTimer &operator=(const KTimer &) = delete;
    ~KTimer() {
        for (auto &r : recs) {
            event_pool_put(r.a);
            event_pool_put(r.b);
        }
    }
    bool timed(int fam) const { return on && ((mask >> fam) & 1u); }  // launches of fam get events
    void begin(int fam, double fl, cudaStream_t s) {
        flops[fam] += fl;
        launches[fam] += 1;
        open = on && ((mask >> fam) & 1u);
        if (!open) return;
        Rec r{fam, event_pool_get(), event_pool_get()};
        cudaEventRecord(r.a, s);
        recs.push_back(r);
    }
    void end(cudaStream_t s) {
        if (open && !recs.empty()) cudaEventRecord(recs.back().b, s);
        open = false;
    }
    // after the stream has been synchronised
    void collect(double ms[GM_K_NFAM]) {
        for (auto &r : recs) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.fam] += t;
            event_pool_put(r.a);
            event_pool_put(r.b);
        }
        recs.clear();
        cudaGetLastError();
    }
};

size_t leaf_smem_bytes(int a, int b);

cudaError_t launch_leaf(const LeafDesc *d_leaves, const std::vector<LeafDesc> &h_leaves, int max_a, int max_b,
                        const double *b, const double *c, const double *d, double *out, Status *st, int stage,
                        cudaStream_t s, KTimer &kt);
cudaError_t launch_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                            double *ws, int nb, int *piv, int piv_ld, double *u12, int64_t u12_stride, Status *st,
                            int stage, cudaStream_t s, KTimer &kt);
cudaError_t launch_merge_assemble(const MergeDesc *md, int nm, const int *tab, const double *in, double *ws,
                                  int64_t max_elems, const double *b, const double *c, const double *d, int n,
                                  cudaStream_t s, KTimer &kt);
// The factored update of an accelerated merge (Section 5, Step 2): rows P1 of the parent
// get L13 W13, rows P2 get L24 W24 (L13: n1 x k13, L24: n2 x k24, column-major with
// leading dimensions n1, n2; W13: k13 x rp, W24: k24 x rp, leading dimensions k13, k24).
struct LrUpdate {
    const double *L13, *L24, *W13, *W24;
    int k13, k24;
};
cudaError_t launch_merge_update_lr(const MergeDesc *md, const MergeDesc &h_md, const int *tab, const double *in,
                                   const LrUpdate &lr, double *out, const double *b, const double *c, const double *d,
                                   cudaStream_t s, KTimer &kt);
cudaError_t launch_merge_update(const MergeDesc *md, const std::vector<MergeDesc> &h_md, const int *tab,
                                const double *in, const double *ws, double *out, int max_rp, const double *b,
                                const double *c, const double *d, int n, cudaStream_t s, KTimer &kt);
cudaError_t launch_root_assemble(const double *S, int r, int n, double *ws, const double *b, const double *c,
                                 const double *d, cudaStream_t s, KTimer &kt);
cudaError_t launch_root_finalize(const double *ws, int r, int n, double *T, cudaStream_t s, KTimer &kt);
cudaError_t launch_apply(const double *T, const double *G, double *V, int N, int B, cudaStream_t s);
// Several dense FP64 applies in one launch (one descriptor per operator; tile0 is filled
// in by the launcher, which uploads the descriptors to d, device memory for h.size()).
struct ApplyDesc {
    const double *T, *G;
    double *V;
    int N, B, tile0, pad;
};
cudaError_t launch_apply_many(std::vector<ApplyDesc> &h, ApplyDesc *d, cudaStream_t s);

}  // namespace gm
