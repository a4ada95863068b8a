// Launchers of the CUDA kernels (host side).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "gm_internal.h"

#define LEAF_THREADS 256
#define GJ_PANEL_THREADS 512
#define GJ_MAX_NB 16

namespace gm {

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
cudaError_t launch_merge_update(const MergeDesc *md, const std::vector<MergeDesc> &h_md, const int *tab,
                                const double *in, const double *ws, double *out, int max_rp, const double *b,
                                const double *c, const double *d, int n, cudaStream_t s, KTimer &kt);
cudaError_t launch_root_assemble(const double *S, int r, int n, double *ws, const double *b, const double *c,
                                 const double *d, cudaStream_t s, KTimer &kt);
cudaError_t launch_root_finalize(const double *ws, int r, int n, double *T, cudaStream_t s, KTimer &kt);
cudaError_t launch_apply(const double *T, const double *G, double *V, int N, int B, cudaStream_t s);

}  // namespace gm
