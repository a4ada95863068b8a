// Launchers of the mixed-precision (df32 storage, split-product tensor-core) build.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "gm_internal.h"
#include "kernels.h"

#define MX_PANEL_THREADS 512

namespace gm {

// Per-stage scratch of the df32 Gauss-Jordan sweep (sized for the largest stage).
struct MxScratch {
    int *perm = nullptr;         // [systems][4 * GJ_MAX_NB]: (destination, source) pairs
    int *perm_n = nullptr;       // [systems]
    float2 *a11inv = nullptr;    // [systems][GJ_MAX_NB * GJ_MAX_NB]: inverse pivot block
    __nv_bfloat16 *fdig = nullptr, *rdig = nullptr;  // digit planes of F (rows) and R (columns)
    int64_t fplane = 0, rplane = 0;                  // plane sizes: 16 * sum of rows / columns
    int *fex = nullptr, *rex = nullptr;              // exponents
};

cudaError_t mx_convert(const double *x, float2 *y, int64_t n, cudaStream_t s, KTimer &kt);
size_t mx_leaf_smem_bytes(int a, int b);
size_t mx_leaf_lines_smem_bytes(int a, int b);
cudaError_t mx_leaf(const LeafDesc *d_leaves, const std::vector<LeafDesc> &h_leaves, int max_a, int max_b,
                    const double *b, const double *c, const double *d, float2 *out, Status *st, int stage,
                    cudaStream_t s, KTimer &kt);
cudaError_t mx_merge_assemble(const MergeDesc *md, int nm, const int *tab, const float2 *in, float2 *ws,
                              int64_t max_elems, const double *b, const double *c, const double *d, int n,
                              cudaStream_t s, KTimer &kt);
cudaError_t mx_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                        float2 *ws, int nb, int split, MxScratch &scr, Status *st, int stage, cudaStream_t s,
                        KTimer &kt);
cudaError_t mx_merge_update(const MergeDesc *md, const std::vector<MergeDesc> &h_md, const int *tab,
                            const float2 *in, const float2 *ws, float2 *out, int max_rp, int split,
                            __nv_bfloat16 *ydig, int *yex, __nv_bfloat16 *xdig, int *xex, int64_t plane,
                            const double *b, const double *c, const double *d, int n, Status *st, cudaStream_t s,
                            KTimer &kt, int wait_limit, int tc_min_k);
cudaError_t mx_root_assemble(const float2 *S, int r, int n, float2 *ws, const double *b, const double *c,
                             const double *d, cudaStream_t s, KTimer &kt);
int mx_kpad(int N);
// T, its df32 copy and T's digit planes from the solved root system; a non-finite entry
// of T sets st->code = GM_ESINGULAR (where = stage).
cudaError_t mx_root_finalize(const float2 *ws, int r, int n, double *T, float2 *Tdf, __nv_bfloat16 *tdig, int *tex,
                             int split, Status *st, int stage, cudaStream_t s, KTimer &kt);
// One operator of a grouped split-product apply: V (N x B, FP64) = T G from T's digit
// planes (tdig, tex: N x kpad per plane, built with the handle) and G (FP64), sliced into
// gdig / gex (gplane elements per plane, at least B * kpad; B exponents).
struct MxApplyDesc {
    const __nv_bfloat16 *tdig;
    const int *tex;
    const double *G;
    double *V;
    __nv_bfloat16 *gdig;
    int *gex;
    int64_t gplane;
    int N, B, kpad, tile0, blk0, pad;
};
// Slices every G and runs every V = T G in two launches (descriptors uploaded to d,
// device memory for h.size(); tile0 and blk0 filled in here).  All share split.
cudaError_t mx_apply_many(std::vector<MxApplyDesc> &h, MxApplyDesc *d, int split, cudaStream_t s);
cudaError_t mx_apply(const __nv_bfloat16 *tdig, const int *tex, const double *G, __nv_bfloat16 *gdig, int *gex,
                     double *V, int N, int B, int split, cudaStream_t s);

}  // namespace gm
