// Mixed-precision build: double-float storage, FP32 pivot search, and the dense
// updates of eq. S_fromtwo_nd on the tensor cores through exact split products.
//
// Storage.  Every Schur complement and every dense system [M | Z] is kept as a
// double-float (df32): an unevaluated sum hi + lo of two FP32 numbers (48-bit
// significand).  All arithmetic outside the tensor cores then runs on the FP32 pipe
// instead of GB300's FP64 pipe (1/64 of the FP32 rate).
//
// Split products.  For C = A B the rows of A and the columns of B are scaled by powers
// of two (row i by 2^-e_i, column j by 2^-f_j, so every scaled entry is below 1 in
// magnitude) and cut into S signed integer digits,
//     x 2^(6-e) = d_0 + 2^-7 d_1 + ... + 2^-7(S-1) d_(S-1) + remainder,  |d_s| <= 64,
// each exactly representable in bf16.  A product of two digits is at most 2^12, so a
// K-long dot product of digits is an integer below 2^24 for K <= 2^12 / (pairs per
// level): the tensor core's FP32 accumulation is then exact.  Pairs (s, t) with
// s + t = g share the scale 2^(-7g) and one accumulator per level g; pairs with
// s + t >= S are dropped.  The epilogue combines the S exact level sums in df32:
//     (A B)_ij ~= 2^(e_i + f_j - 12) sum_g acc_g 2^(-7g).
// The digit products use mma.sync m16n8k16 (bf16 in, FP32 accumulate).
//
// Gauss-Jordan sweep with FP32 pivot search.  Per panel of nb columns the pivot rows
// are chosen by partial pivoting on an FP32 copy of the panel; the chosen rows move to
// the pivot positions (row interchanges on the df32 data), the pivot block A11 is
// factored without further interchanges, R = A11^{-1} A12 is written into the pivot
// rows, and every other row i takes  row_i -= A(i, panel) R  with A(i, panel) its
// values at the start of the step.  For rows below the panel this equals the usual
// L21 U12 update; for rows above it eliminates their panel entries, so at the end the
// right block holds M^{-1} Z.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gm_internal.h"
#include "kernels.h"
#include "mixed.h"
#include "mixed_dev.cuh"

namespace gm {

// ----------------------------------------------------------------------------- conversions

__global__ void k_mx_d2df(const double *__restrict__ x, float2 *__restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = df_from_d(x[i]);
}

// ----------------------------------------------------------------------------- merge assemble

// [M | Z] (df32) with M = [S33 A34; A43 S44], Z = [S31 0; 0 S42].
__global__ void __launch_bounds__(256)
k_mx_merge_assemble(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const float2 *__restrict__ in,
                    float2 *__restrict__ ws, const double *__restrict__ bf, const double *__restrict__ cf,
                    const double *__restrict__ df, int n) {
    const MergeDesc M = md[blockIdx.y];
    const MergeTabMx T = merge_tab_mx(M, tab);
    const int sp = M.sp, mm = 2 * sp, ncol = mm + M.rp;
    const int64_t tot = (int64_t)mm * ncol;
    const float2 *S1 = in + M.s1, *S2 = in + M.s2;
    float2 *A = ws + M.ws;
    const double ih = M.n + 1.0;  // 1/h of the merge's problem
    const int d34 = M.orient ? DIR_N : DIR_E, d43 = M.orient ? DIR_S : DIR_W;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int t = (int)(e % mm), c = (int)(e / mm);
        float2 v = make_float2(0.f, 0.f);
        if (c < mm) {
            if (t < sp && c < sp) v = S1[T.p3[t] + (int64_t)M.r1 * T.p3[c]];
            else if (t >= sp && c >= sp) v = S2[T.p4[t - sp] + (int64_t)M.r2 * T.p4[c - sp]];
            else if (t < sp) { if (c - sp == t) v = df_from_d(stencil_w_mx(bf, cf, df, ih, T.g3[t], d34)); }
            else if (c == t - sp) v = df_from_d(stencil_w_mx(bf, cf, df, ih, T.g4[t - sp], d43));
        } else {
            int cc = c - mm;
            if (cc < M.n1) { if (t < sp) v = S1[T.p3[t] + (int64_t)M.r1 * T.p1[cc]]; }
            else if (t >= sp) v = S2[T.p4[t - sp] + (int64_t)M.r2 * T.p2[cc - M.n1]];
        }
        A[e] = v;
    }
}

// ----------------------------------------------------------------------------- GJ sweep (df32)

// Panel: FP32 partial pivoting on the hi parts of rows k..m-1 of columns k..k+nbe-1
// chooses the pivot rows; their composed row interchanges are applied to the panel
// columns (df32); the pivot block A11 is factored and inverted in FP64; A11^{-1} is
// stored as df32 for the pivot-row kernel.
// perm[sys]: up to 2nb (destination, source) row pairs, count in perm_n[sys].
__global__ void __launch_bounds__(MX_PANEL_THREADS)
k_mx_gj_panel(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int nb, int *__restrict__ perm,
              int *__restrict__ perm_n, float2 *__restrict__ a11inv, Status *st, int stage) {
    extern __shared__ float smf[];
    __shared__ float s_val[32];
    __shared__ int s_idx[32];
    __shared__ int s_piv[GJ_MAX_NB];
    __shared__ int s_src[2 * GJ_MAX_NB], s_dst[2 * GJ_MAX_NB], s_cnt;
    __shared__ double s_lu[GJ_MAX_NB][GJ_MAX_NB + 1];
    __shared__ double s_inv[GJ_MAX_NB][GJ_MAX_NB + 1];
    const SysDesc S = sys[blockIdx.x];
    const int m = S.m;
    if (k >= m) return;
    const int nbe = min(nb, m - k), rows = m - k;
    float2 *A = ws + S.off;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    float *P = smf;  // rows x nbe, column-major, hi parts
    for (int e = tid; e < rows * nbe; e += nt) {
        int rr = e % rows, c = e / rows;
        P[(size_t)c * rows + rr] = A[(size_t)(k + c) * m + k + rr].x;
    }
    __syncthreads();
    for (int t = 0; t < nbe; ++t) {
        float best = -1.f;
        int bi = 0x7fffffff;
        for (int rr = t + tid; rr < rows; rr += nt) {
            float v = fabsf(P[(size_t)t * rows + rr]);
            if (v > best) { best = v; bi = rr; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            float v2 = __shfl_down_sync(0xffffffffu, best, o);
            int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (wid == 0) {
            best = lane < nw ? s_val[lane] : -1.f;
            bi = lane < nw ? s_idx[lane] : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                float v2 = __shfl_down_sync(0xffffffffu, best, o);
                int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
            }
            if (lane == 0) {
                if (bi < t || bi >= rows) bi = t;  // no finite candidate: keep the diagonal
                s_idx[0] = bi;
                s_piv[t] = bi;
            }
        }
        __syncthreads();
        const int pr = s_idx[0];
        if (pr != t)
            for (int c = tid; c < nbe; c += nt) {
                float x = P[(size_t)c * rows + t];
                P[(size_t)c * rows + t] = P[(size_t)c * rows + pr];
                P[(size_t)c * rows + pr] = x;
            }
        __syncthreads();
        const float pv = P[(size_t)t * rows + t];
        const float inv = pv != 0.f ? 1.f / pv : 0.f;
        for (int rr = t + 1 + tid; rr < rows; rr += nt) {
            float l = P[(size_t)t * rows + rr] * inv;
            P[(size_t)t * rows + rr] = l;
            for (int c = t + 1; c < nbe; ++c) P[(size_t)c * rows + rr] -= l * P[(size_t)c * rows + t];
        }
        __syncthreads();
    }
    // compose the interchanges: new position r takes the row that was at src(r)
    if (tid == 0) {
        int pos[2 * GJ_MAX_NB], who[2 * GJ_MAX_NB], cnt = 0;
        for (int t = 0; t < nbe; ++t) {
            int a = -1, b = -1;
            for (int i = 0; i < cnt; ++i) {
                if (pos[i] == t) a = i;
                if (pos[i] == s_piv[t]) b = i;
            }
            if (a < 0) { pos[cnt] = t; who[cnt] = t; a = cnt++; }
            if (b < 0) { pos[cnt] = s_piv[t]; who[cnt] = s_piv[t]; b = cnt++; }
            int x = who[a]; who[a] = who[b]; who[b] = x;
        }
        for (int i = 0; i < cnt; ++i) { s_dst[i] = k + pos[i]; s_src[i] = k + who[i]; }
        s_cnt = cnt;
        perm_n[blockIdx.x] = cnt;
        for (int i = 0; i < cnt; ++i) {
            perm[(size_t)blockIdx.x * 4 * GJ_MAX_NB + 2 * i] = k + pos[i];
            perm[(size_t)blockIdx.x * 4 * GJ_MAX_NB + 2 * i + 1] = k + who[i];
        }
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int c = tid; c < nbe; c += nt) {
        float2 *col = A + (size_t)(k + c) * m;
        float2 vals[2 * GJ_MAX_NB];
        for (int i = 0; i < cnt; ++i) vals[i] = col[s_src[i]];
        for (int i = 0; i < cnt; ++i) col[s_dst[i]] = vals[i];
    }
    __syncthreads();
    // FP64 LU (no further interchanges) and inverse of the pivot block A11
    for (int e = tid; e < nbe * nbe; e += nt) {
        int i = e % nbe, j = e / nbe;
        s_lu[i][j] = df_to_d(A[(size_t)(k + j) * m + k + i]);
    }
    __syncthreads();
    double minp = 1e300;
    for (int t = 0; t < nbe; ++t) {
        const double pv = s_lu[t][t];
        minp = fmin(minp, fabs(pv));
        if (!(fabs(pv) > 0.0) || !isfinite(pv)) {
            if (tid == 0) record_pivot_mx(st + S.prob, pv, stage);
        }
        for (int i = t + 1 + tid; i < nbe; i += nt) s_lu[i][t] = s_lu[i][t] / pv;
        __syncthreads();
        const int w = nbe - t - 1;
        for (int e = tid; e < w * w; e += nt) {
            int i = t + 1 + e / w, j = t + 1 + e % w;
            s_lu[i][j] -= s_lu[i][t] * s_lu[t][j];
        }
        __syncthreads();
    }
    if (tid == 0 && minp > 0.0 && minp < 1e300) record_pivot_mx(st + S.prob, minp, stage);
    if (tid < nbe) {  // column tid of A11^{-1}: L y = e_tid, U x = y
        double x[GJ_MAX_NB];
        for (int i = 0; i < nbe; ++i) {
            double sacc = (i == tid) ? 1.0 : 0.0;
            for (int q = 0; q < i; ++q) sacc -= s_lu[i][q] * x[q];
            x[i] = sacc;
        }
        for (int i = nbe - 1; i >= 0; --i) {
            double sacc = x[i];
            for (int q = i + 1; q < nbe; ++q) sacc -= s_lu[i][q] * x[q];
            x[i] = sacc / s_lu[i][i];
        }
        for (int i = 0; i < nbe; ++i) s_inv[i][tid] = x[i];
    }
    __syncthreads();
    for (int e = tid; e < nbe * nbe; e += nt) {
        int i = e / nbe, j = e % nbe;
        a11inv[(size_t)blockIdx.x * GJ_MAX_NB * GJ_MAX_NB + i * GJ_MAX_NB + j] = df_from_d(s_inv[i][j]);
    }
}

// Per step, after the panel.  Blocks [0, cb) take 128 columns right of the panel each:
// apply the composed interchanges, R = A11^{-1} A12 (df32), write R into the pivot rows
// and slice it (digit planes of the column operand).  Blocks [cb, cb + rb) take 128
// rows each and slice F = A(i, panel) (zero for the pivot rows) as the row operand.
template <int S>
__global__ void __launch_bounds__(128)
k_mx_gj_prep(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int nb, int cb,
             const int *__restrict__ perm, const int *__restrict__ perm_n, const float2 *__restrict__ a11inv,
             __nv_bfloat16 *__restrict__ fdig, int64_t fplane, int *__restrict__ fex, __nv_bfloat16 *__restrict__ rdig,
             int64_t rplane, int *__restrict__ rex) {
    __shared__ float2 Ai[GJ_MAX_NB][GJ_MAX_NB + 1];
    __shared__ int s_src[2 * GJ_MAX_NB], s_dst[2 * GJ_MAX_NB];
    const SysDesc Sy = sys[blockIdx.y];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(nb, m - k);
    float2 *A = ws + Sy.off;
    if ((int)blockIdx.x >= cb) {  // row operand F
        const int i = ((int)blockIdx.x - cb) * 128 + threadIdx.x;
        if (i >= m) return;
        const bool piv = i >= k && i < k + nbe;
        float2 v[GJ_MAX_NB];
        float mx = 0.f;
#pragma unroll
        for (int t = 0; t < GJ_MAX_NB; ++t) {
            v[t] = (t < nbe && !piv) ? A[(size_t)(k + t) * m + i] : make_float2(0.f, 0.f);
            mx = fmaxf(mx, fabsf(v[t].x));
        }
        const int e = exp_of_max(mx * 1.0000001f);
        const int64_t row = Sy.roff + i;
        fex[row] = e;
#pragma unroll
        for (int t = 0; t < GJ_MAX_NB; ++t) {
            float d[S];
            digits<S>(v[t], e, d);
#pragma unroll
            for (int s = 0; s < S; ++s) fdig[(int64_t)s * fplane + row * 16 + t] = __float2bfloat16_rn(d[s]);
        }
        return;
    }
    const int cnt = perm_n[blockIdx.y];
    for (int e = threadIdx.x; e < nbe * nbe; e += blockDim.x) {
        int i = e / nbe, j = e % nbe;
        Ai[i][j] = a11inv[(size_t)blockIdx.y * GJ_MAX_NB * GJ_MAX_NB + i * GJ_MAX_NB + j];
    }
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        s_dst[e] = perm[(size_t)blockIdx.y * 4 * GJ_MAX_NB + 2 * e];
        s_src[e] = perm[(size_t)blockIdx.y * 4 * GJ_MAX_NB + 2 * e + 1];
    }
    __syncthreads();
    const int j = k + nbe + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Sy.ncol) return;
    float2 *col = A + (size_t)j * m;
    {
        float2 vals[2 * GJ_MAX_NB];
        for (int i = 0; i < cnt; ++i) vals[i] = col[s_src[i]];
        for (int i = 0; i < cnt; ++i) col[s_dst[i]] = vals[i];
    }
    float2 a12[GJ_MAX_NB], r[GJ_MAX_NB];
#pragma unroll
    for (int t = 0; t < GJ_MAX_NB; ++t) a12[t] = t < nbe ? col[k + t] : make_float2(0.f, 0.f);
    float mx = 0.f;
#pragma unroll
    for (int t = 0; t < GJ_MAX_NB; ++t) {
        float2 acc = make_float2(0.f, 0.f);
        if (t < nbe)
#pragma unroll
            for (int q = 0; q < GJ_MAX_NB; ++q)
                if (q < nbe) acc = df_add(acc, df_mul(Ai[t][q], a12[q]));
        r[t] = acc;
        if (t < nbe) col[k + t] = acc;
        mx = fmaxf(mx, fabsf(acc.x));
    }
    const int e = exp_of_max(mx * 1.0000001f);
    const int64_t row = Sy.coff + j;
    rex[row] = e;
#pragma unroll
    for (int t = 0; t < GJ_MAX_NB; ++t) {
        float d[S];
        digits<S>(r[t], e, d);
#pragma unroll
        for (int s = 0; s < S; ++s) rdig[(int64_t)s * rplane + row * 16 + t] = __float2bfloat16_rn(d[s]);
    }
}

// Rank-nbe update of every non-pivot row on the tensor cores from the sliced F and R:
//   A(i, j) -= sum_t F(i, t) R(t, j),  64 x 64 tile per CTA.
template <int S>
__global__ void __launch_bounds__(128)
k_mx_gj_update(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int nb,
               const __nv_bfloat16 *__restrict__ fdig, int64_t fplane, const int *__restrict__ fex,
               const __nv_bfloat16 *__restrict__ rdig, int64_t rplane, const int *__restrict__ rex) {
    __shared__ __align__(16) __nv_bfloat16 As[S * 64 * KP];
    __shared__ __align__(16) __nv_bfloat16 Bs[S * 64 * KP];
    const SysDesc Sy = sys[blockIdx.z];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(nb, m - k);
    const int i0 = blockIdx.x * 64, j0 = k + nbe + blockIdx.y * 64;
    if (i0 >= m || j0 >= Sy.ncol) return;
    float2 *A = ws + Sy.off;
    digit_gemm_chunks<S>(fdig + (int64_t)Sy.roff * 16, fplane, 16, i0, m, fex + Sy.roff, rdig + (int64_t)Sy.coff * 16,
                         rplane, 16, j0, Sy.ncol, rex + Sy.coff, 16, As, Bs,
                         [&](const int *r, const int *cl, const float2 *v, bool) {
                             float2 w[4];
                             bool ok[4];
#pragma unroll
                             for (int q = 0; q < 4; ++q) {
                                 const int i = i0 + r[q], j = j0 + cl[q];
                                 ok[q] = !(i >= m || j >= Sy.ncol || (i >= k && i < k + nbe));
                                 w[q] = ok[q] ? A[(size_t)j * m + i] : make_float2(0.f, 0.f);
                             }
#pragma unroll
                             for (int q = 0; q < 4; ++q)
                                 if (ok[q]) A[(size_t)(j0 + cl[q]) * m + i0 + r[q]] = df_sub(w[q], v[q]);
                         });
}

// ----------------------------------------------------------------------------- merge update

// Slice the Schur-update operands of every merge of a stage:
//   rows a of Y' = [S13 0; 0 S24] (rp x 2sp) and columns c of X = M^{-1} Z (2sp x rp).
// One warp per row (blockIdx.x < rb * 4 warps) or per column.
template <int S>
__global__ void __launch_bounds__(128)
k_mx_merge_slice(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const float2 *__restrict__ in,
                 const float2 *__restrict__ ws, int rb, __nv_bfloat16 *__restrict__ ydig, int *__restrict__ yex,
                 __nv_bfloat16 *__restrict__ xdig, int *__restrict__ xex, int64_t plane, int tiled) {
    const MergeDesc M = md[blockIdx.y];
    const MergeTabMx T = merge_tab_mx(M, tab);
    const int sp = M.sp, mm = 2 * sp, n1 = M.n1, warp = threadIdx.x >> 5;
    const bool rows = (int)blockIdx.x < rb;
    const int idx = ((rows ? (int)blockIdx.x : (int)blockIdx.x - rb) * 4) + warp;
    if (idx >= M.rp) return;
    if (rows) {
        const float2 *S1 = in + M.s1, *S2 = in + M.s2;
        const int a = idx;
        auto get = [&](int kk) -> float2 {
            if (a < n1) return kk < sp ? S1[T.p1[a] + (int64_t)M.r1 * T.p3[kk]] : make_float2(0.f, 0.f);
            return kk >= sp ? S2[T.p2[a - n1] + (int64_t)M.r2 * T.p4[kk - sp]] : make_float2(0.f, 0.f);
        };
        warp_slice_row<S>(get, mm, M.kpad, ydig + M.doff, plane, a, yex + M.eoff, tiled != 0);
    } else {
        const float2 *X = ws + M.ws + (size_t)mm * mm;
        const int c = idx;
        auto get = [&](int kk) -> float2 { return X[(size_t)c * mm + kk]; };
        warp_slice_row<S>(get, mm, M.kpad, xdig + M.doff, plane, c, xex + M.eoff, tiled != 0);
    }
}

// S_parent(q(a), q(c)) = C(a, c) - (Y' X)(a, c), C = [S11 A12; A21 S22].
template <int S>
__global__ void __launch_bounds__(PIPE_THREADS)
k_mx_merge_update(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const float2 *__restrict__ in,
                  float2 *__restrict__ out, const __nv_bfloat16 *__restrict__ ydig, const int *__restrict__ yex,
                  const __nv_bfloat16 *__restrict__ xdig, const int *__restrict__ xex, int64_t plane,
                  const double *__restrict__ bf, const double *__restrict__ cf, const double *__restrict__ df, int n) {
    extern __shared__ __align__(16) unsigned char smem_raw[];  // pipe_smem_bytes(S)
    const MergeDesc M = md[blockIdx.z];
    const int rp = M.rp;
    const int a0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
    if (a0 >= rp || c0 >= rp) return;
    const MergeTabMx T = merge_tab_mx(M, tab);
    const int n1 = M.n1;
    const float2 *S1 = in + M.s1, *S2 = in + M.s2;
    const int64_t eo = M.eoff;
    const double ih = M.n + 1.0;  // 1/h of the merge's problem
    const int d12 = M.orient ? DIR_N : DIR_E, d21 = M.orient ? DIR_S : DIR_W;
    float2 *O = out + M.out;
    digit_gemm_pipe<S>(
        ydig + M.doff, plane, M.kpad, a0, rp, yex + eo, xdig + M.doff, plane, M.kpad, c0, rp, xex + eo, 2 * M.sp,
        (__nv_bfloat16 *)smem_raw,
        [&](const int *r, const int *cl, const float2 *v, bool first) {
            // the four parent positions and their current values (children's entries on
            // the first chunk, the partial result after), read together
            float2 cval[4];
            int64_t off[4];
            bool ok[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int aa = a0 + r[q], cc = c0 + cl[q];
                ok[q] = aa < rp && cc < rp;
                cval[q] = make_float2(0.f, 0.f);
                off[q] = 0;
                if (!ok[q]) continue;
                const int qa = aa < n1 ? T.q1[aa] : T.q2[aa - n1];
                const int qc = cc < n1 ? T.q1[cc] : T.q2[cc - n1];
                off[q] = qa + (int64_t)rp * qc;
                if (!first) {  // a later K chunk: accumulate into the parent entry
                    cval[q] = O[off[q]];
                } else if (aa < n1 && cc < n1) {
                    cval[q] = S1[T.p1[aa] + (int64_t)M.r1 * T.p1[cc]];
                } else if (aa >= n1 && cc >= n1) {
                    cval[q] = S2[T.p2[aa - n1] + (int64_t)M.r2 * T.p2[cc - n1]];
                } else {
                    for (int e = 0; e < 2; ++e) {
                        const int *x = T.x12 + 4 * e;
                        if (aa < n1 && aa == x[0] && cc - n1 == x[1])
                            cval[q] = df_from_d(stencil_w_mx(bf, cf, df, ih, x[2], d12));
                        if (aa >= n1 && aa - n1 == x[1] && cc == x[0])
                            cval[q] = df_from_d(stencil_w_mx(bf, cf, df, ih, x[3], d21));
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (ok[q]) O[off[q]] = df_sub(cval[q], v[q]);
        });
}

// ----------------------------------------------------------------------------- merge update, tcgen05

// The same S_parent(q(a), q(c)) = C(a, c) - (Y' X)(a, c) on the fifth-generation tensor
// cores: a CTA takes 128 rows (a) x 64 columns (c) of the parent; the 16-k digit tiles of
// Y and X stream through four shared-memory stages by bulk copies on the tensor memory
// accelerator (one 4 KB / 2 KB copy per digit plane, counted on the stage's `full`
// barrier, issued by a producer thread); another thread issues each tile's 21 digit-pair
// products as tcgen05.mma
// (M = 128, N = 64, K = 16) into six level accumulators in tensor memory and commits
// them to the stage's `empty` barrier, and a stage is refilled only once that commit
// has landed.  K runs in chunks of at most 512: level g sums g + 1 digit pairs of at most
// 64 x 64 each, and (g + 1) 512 64^2 < 2^24 for g < 6, so every level sum is exact in fp32;
// after each chunk eight warps read the levels back (tcgen05.ld) and apply the same
// epilogue as the mma.sync kernel.  Every wait is bounded (GM_ETIMEOUT, no hang).
constexpr int MT_ROWS = 128, MT_COLS = 64, MT_STAGES = 4, MT_KTILES = 32;  // 32 x 16 = 512 k per chunk

size_t mx_merge_tc_smem(int split) {
    // at least 120 KB, so one CTA per SM: each CTA allocates all 512 tensor-memory columns
    const size_t need = (size_t)MT_STAGES * split * (MT_ROWS + MT_COLS) * 16 * sizeof(__nv_bfloat16) + 1024;
    return need > 120 * 1024 ? need : 120 * 1024;
}

// Tile layout in a stage: A rows a0 .. a0 + 127 first, then B rows c0 .. c0 + 63; plane q
// of A at q * 4096, of B at S * 4096 + q * 2048; core matrix (row / 8, k / 8) of a 16-k
// tile at (row / 8) 256 + (k / 8) 128 -- the order the digit planes are stored in (rows
// padded to 128; padding rows only reach outputs that are never stored).
template <int S>
__global__ void __launch_bounds__(PIPE_THREADS)
k_mx_merge_update_tc(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const float2 *__restrict__ in,
                     float2 *__restrict__ out, const __nv_bfloat16 *__restrict__ ydig, const int *__restrict__ yex,
                     const __nv_bfloat16 *__restrict__ xdig, const int *__restrict__ xex, int64_t plane,
                     const double *__restrict__ bf, const double *__restrict__ cf, const double *__restrict__ df,
                     Status *__restrict__ st, int limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int STAGE = S * (MT_ROWS + MT_COLS) * 32;  // bytes per stage
    __shared__ __align__(8) unsigned long long full[MT_STAGES], empty[MT_STAGES];
    __shared__ uint32_t s_tmem;
    __shared__ int s_ye[MT_ROWS], s_xe[MT_COLS];
    __shared__ int s_bad;
    __shared__ int s_loaded, s_committed;  // tiles of the current chunk copied / committed
    const MergeDesc M = md[blockIdx.z];
    const int rp = M.rp;
    const int a0 = blockIdx.x * MT_ROWS, c0 = blockIdx.y * MT_COLS;
    if (a0 >= rp || c0 >= rp) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const MergeTabMx T = merge_tab_mx(M, tab);
    const int n1 = M.n1;
    const float2 *S1 = in + M.s1, *S2 = in + M.s2;
    const double ih = M.n + 1.0;
    const int d12 = M.orient ? DIR_N : DIR_E, d21 = M.orient ? DIR_S : DIR_W;
    float2 *O = out + M.out;
    const int kpad = M.kpad, ntile = kpad / 16;
    // tile-ordered digit planes: the 128-row block of a0 and of c0 (c0's 64 rows are the
    // first or second half of its block)
    const __nv_bfloat16 *Ab = ydig + M.doff + (int64_t)(a0 >> 7) * (kpad >> 4) * 2048;
    const __nv_bfloat16 *Bb = xdig + M.doff + (int64_t)(c0 >> 7) * (kpad >> 4) * 2048 + ((c0 & 127) >> 3) * 128;
    if (tid < MT_ROWS) s_ye[tid] = yex[M.eoff + min(a0 + tid, rp - 1)];
    else if (tid < MT_ROWS + MT_COLS) s_xe[tid - MT_ROWS] = xex[M.eoff + min(c0 + tid - MT_ROWS, rp - 1)];
    if (tid == 0) {
        for (int q = 0; q < MT_STAGES; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[q])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[q])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        s_bad = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = umma_idesc_bf16(MT_ROWS, MT_COLS);
    const int q4 = warp & 3, h = warp >> 2;
    const int aa = a0 + 32 * q4 + lane;  // this thread's parent row in the epilogue
    // 16-k tile t into a stage: one bulk copy per plane of A (4 KB) and of B (2 KB), all
    // counted on the stage's `full` barrier (thread 0 only)
    auto load_tile = [&](int t, int sg) {
        unsigned char *sa = base + sg * STAGE, *sb = sa + S * 4096;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(&full[sg])),
                     "r"((uint32_t)(S * 6144)));
#pragma unroll
        for (int q = 0; q < S; ++q) {
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 4096, [%2];\n" ::"r"(
                             smem_u32(sa + q * 4096)),
                         "l"(Ab + (int64_t)q * plane + (int64_t)t * 2048), "r"(smem_u32(&full[sg])));
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 2048, [%2];\n" ::"r"(
                             smem_u32(sb + q * 2048)),
                         "l"(Bb + (int64_t)q * plane + (int64_t)t * 2048), "r"(smem_u32(&full[sg])));
        }
    };
    // descriptors of stage 0's first planes (a stage or plane offset adds to the address
    // field, which stays below 2^14 units of 16 bytes)
    const uint64_t adesc0 = umma_desc(smem_u32(base), 128, 256), bdesc0 = umma_desc(smem_u32(base + S * 4096), 128, 256);
    // completion parity of the stages' barriers at the start of a chunk (bit s): tile kt of
    // the chunk is completion (chunk base + kt / MT_STAGES) of stage kt % MT_STAGES, for
    // `full` and `empty` alike (each completes once per tile on its stage)
    unsigned bpar = 0u;
    bool bad = false;
    for (int t0 = 0; t0 < ntile && !bad; t0 += MT_KTILES) {
        const int nk = min(ntile - t0, MT_KTILES);
        const bool first = t0 == 0;
        const unsigned bpar0 = bpar;
        if (tid == 32) {  // producer: copies, each stage refilled once its products landed
            int nl = 0;
            for (int t = 0; t < nk && !bad; ++t) {
                const int sg = t % MT_STAGES;
                if (t >= MT_STAGES &&
                    !mbar_wait_bounded(&empty[sg], ((bpar >> sg) & 1u) ^ (uint32_t)((t / MT_STAGES - 1) & 1), limit)) {
                    bad = true;
                } else {
                    load_tile(t0 + t, sg);
                    ++nl;
                }
            }
            s_loaded = nl;
            if (bad) s_bad = 1;
        } else if (tid == 0) {  // products: wait for a stage's copies, issue, commit
            int nc = 0;
            for (int kt = 0; kt < nk; ++kt) {
                const int sg = kt % MT_STAGES;
                if (!mbar_wait_bounded(&full[sg], ((bpar >> sg) & 1u) ^ (uint32_t)((kt / MT_STAGES) & 1), limit)) {
                    bad = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
                const uint64_t da = adesc0 + (uint64_t)((sg * STAGE) >> 4), db = bdesc0 + (uint64_t)((sg * STAGE) >> 4);
#pragma unroll
                for (int a = 0; a < S; ++a)
#pragma unroll
                    for (int b = 0; b < S - a; ++b)
                        umma_bf16(tmem + (uint32_t)((a + b) * MT_COLS), da + (uint64_t)(a * 4096 >> 4),
                                  db + (uint64_t)(b * 2048 >> 4), idesc, (kt > 0 || a > 0) ? 1u : 0u);
                umma_commit(&empty[sg]);
                ++nc;
            }
            s_committed = nc;
            if (bad) s_bad = 1;
        }
        if (warp < 2) __syncwarp();
        // everyone: the chunk's last products (they complete in order)
        const int sl = (nk - 1) % MT_STAGES;
        if (!mbar_wait_bounded(&empty[sl], ((bpar >> sl) & 1u) ^ (uint32_t)(((nk - 1) / MT_STAGES) & 1), limit))
            s_bad = 1;
#pragma unroll
        for (int q = 0; q < MT_STAGES; ++q)  // tiles of this chunk on stage q
            if (q < nk) bpar ^= (uint32_t)(((nk - q + MT_STAGES - 1) / MT_STAGES) & 1) << q;
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        if (s_bad) {
            // gave up: before the tensor memory is released, wait (bounded) for the products
            // committed (they complete in order: the last one suffices) and for the copies
            // issued but not yet consumed (at most one per stage)
            if (tid == 0) {
                const int nc = s_committed, nl = s_loaded;
                if (nc > 0) {
                    const int c = nc - 1, sg = c % MT_STAGES;
                    mbar_wait_bounded(&empty[sg], ((bpar0 >> sg) & 1u) ^ (uint32_t)((c / MT_STAGES) & 1), DRAIN_POLLS);
                }
                for (int t = nc; t < nl; ++t) {
                    const int sg = t % MT_STAGES;
                    mbar_wait_bounded(&full[sg], ((bpar0 >> sg) & 1u) ^ (uint32_t)((t / MT_STAGES) & 1), DRAIN_POLLS);
                }
            }
            bad = true;
            break;
        }
        // epilogue: this thread's row aa, columns c0 + 32 h .. + 31, eight at a time
#pragma unroll 1
        for (int cc0 = 0; cc0 < 32; cc0 += 8) {
            uint32_t v[S][8];
#pragma unroll
            for (int g = 0; g < S; ++g)
                tmem_ld8(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(g * MT_COLS + 32 * h + cc0), v[g]);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
            if (aa >= rp) continue;
            const int qa = aa < n1 ? T.q1[aa] : T.q2[aa - n1];
            float2 cval[8];
            int64_t off[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {  // the eight parent entries' current values, read together
                const int cc = c0 + 32 * h + cc0 + c;
                cval[c] = make_float2(0.f, 0.f);
                off[c] = -1;
                if (cc >= rp) continue;
                const int qc = cc < n1 ? T.q1[cc] : T.q2[cc - n1];
                off[c] = qa + (int64_t)rp * qc;
                if (!first) {
                    cval[c] = O[off[c]];
                } else if (aa < n1 && cc < n1) {
                    cval[c] = S1[T.p1[aa] + (int64_t)M.r1 * T.p1[cc]];
                } else if (aa >= n1 && cc >= n1) {
                    cval[c] = S2[T.p2[aa - n1] + (int64_t)M.r2 * T.p2[cc - n1]];
                } else {
                    for (int e = 0; e < 2; ++e) {
                        const int *x = T.x12 + 4 * e;
                        if (aa < n1 && aa == x[0] && cc - n1 == x[1])
                            cval[c] = df_from_d(stencil_w_mx(bf, cf, df, ih, x[2], d12));
                        if (aa >= n1 && aa - n1 == x[1] && cc == x[0])
                            cval[c] = df_from_d(stencil_w_mx(bf, cf, df, ih, x[3], d21));
                    }
                }
            }
            const int ea = s_ye[32 * q4 + lane];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (off[c] < 0) continue;
                float2 x = make_float2(__uint_as_float(v[S - 1][c]) * pow2f(-7 * (S - 1)), 0.f);
#pragma unroll
                for (int g = S - 2; g >= 0; --g) x = df_add_f(x, __uint_as_float(v[g][c]) * pow2f(-7 * g));
                O[off[c]] = df_sub(cval[c], df_scale(x, ea + s_xe[32 * h + cc0 + c] - 12));
            }
        }
        // the next chunk's products overwrite the accumulators: every read must be done
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    }
    if (bad && tid == 0 && atomicCAS(&st[M.prob].code, 0, GM_ETIMEOUT) == 0) st[M.prob].where = -1;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
}

// ----------------------------------------------------------------------------- root

__device__ __forceinline__ void ghost_nb_mx(int n, int k, int &g, int &dir) {
    int side = k / n, t = k % n;
    if (side == 0) { g = t; dir = DIR_S; }
    else if (side == 1) { g = (n - 1) + n * t; dir = DIR_E; }
    else if (side == 2) { g = (n - 1 - t) + n * (n - 1); dir = DIR_N; }
    else { g = n * (n - 1 - t); dir = DIR_W; }
}
__device__ __forceinline__ int ghost_ring_mx(int n, int k) {
    int r = 4 * n - 4;
    int p = k - k / n;
    return p >= r ? p - r : p;
}

__global__ void k_mx_root_assemble(const float2 *__restrict__ S, int r, int n, float2 *__restrict__ ws,
                                   const double *__restrict__ bf, const double *__restrict__ cf,
                                   const double *__restrict__ df) {
    const int64_t tot = (int64_t)r * (r + 4 * n);
    const double ih = n + 1.0;  // 1/h
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int row = (int)(e % r), c = (int)(e / r);
        float2 v = make_float2(0.f, 0.f);
        if (c < r) v = S[e];
        else {
            int k = c - r, g, dir;
            ghost_nb_mx(n, k, g, dir);
            if (row == ghost_ring_mx(n, k)) v = df_from_d(-stencil_w_mx(bf, cf, df, ih, g, dir));
        }
        ws[e] = v;
    }
}

// T[k, k'] = (delta - X[ring(k), k']) (n+1): FP64 for the user, df32 for the apply.
// A non-finite entry of T (a Schur complement that left the double-float range, which is
// FP32's, on the way) is reported like a non-finite pivot: GM_ESINGULAR at the root stage,
// so that the automatic mode rebuilds the problem in FP64.
__global__ void k_mx_root_finalize(const float2 *__restrict__ ws, int r, int n, double *__restrict__ T,
                                   float2 *__restrict__ Tdf, Status *__restrict__ st, int stage) {
    const int nb4 = 4 * n;
    const int64_t tot = (int64_t)nb4 * nb4;
    const float2 *X = ws + (size_t)r * r;
    const float inv_h = (float)(n + 1);  // exact for n < 2^24
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(e % nb4), kp = (int)(e / nb4);
        float2 x = X[(size_t)kp * r + ghost_ring_mx(n, k)];
        float2 v = df_sub(make_float2(k == kp ? 1.f : 0.f, 0.f), x);
        v = df_mul(v, make_float2(inv_h, 0.f));
        Tdf[e] = v;
        T[e] = df_to_d(v);
        bad |= !isfinite(v.x) || !isfinite(v.y);
    }
    if (bad && st && atomicCAS(&st->code, 0, GM_ESINGULAR) == 0) st->where = stage;
}

// ----------------------------------------------------------------------------- apply

// Slice the rows of T (N x N column-major df32) once per build: warp per row.
template <int S>
__global__ void __launch_bounds__(128)
k_mx_slice_T(const float2 *__restrict__ Tdf, int N, int kpad, __nv_bfloat16 *__restrict__ dig, int64_t plane,
             int *__restrict__ ex) {
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (i >= N) return;
    auto get = [&](int j) -> float2 { return Tdf[(size_t)j * N + i]; };
    warp_slice_row<S>(get, N, kpad, dig, plane, i, ex);
}

// Slice the columns of G (N x B column-major FP64) per solve: warp per column.
template <int S>
__global__ void __launch_bounds__(128)
k_mx_slice_G(const double *__restrict__ G, int N, int B, int kpad, __nv_bfloat16 *__restrict__ dig, int64_t plane,
             int *__restrict__ ex) {
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (j >= B) return;
    auto get = [&](int kk) -> float2 { return df_from_d(G[(size_t)j * N + kk]); };
    warp_slice_row<S>(get, N, kpad, dig, plane, j, ex);
}

// V = T G from the sliced operands; V is FP64 N x B.
template <int S>
__global__ void __launch_bounds__(PIPE_THREADS)
k_mx_apply(const __nv_bfloat16 *__restrict__ tdig, const int *__restrict__ tex, int64_t tplane,
           const __nv_bfloat16 *__restrict__ gdig, const int *__restrict__ gex, int64_t gplane, int kpad,
           double *__restrict__ V, int N, int B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];  // pipe_smem_bytes(S)
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    digit_gemm_pipe<S>(tdig, tplane, kpad, i0, N, tex, gdig, gplane, kpad, j0, B, gex, N, (__nv_bfloat16 *)smem_raw,
                         [&](const int *r, const int *cl, const float2 *v, bool first) {
#pragma unroll
                             for (int q = 0; q < 4; ++q) {
                                 const int i = i0 + r[q], j = j0 + cl[q];
                                 if (i >= N || j >= B) continue;
                                 double *o = V + (size_t)j * N + i;
                                 *o = first ? df_to_d(v[q]) : *o + df_to_d(v[q]);
                             }
                         });
}

// Several split-product applies in one pair of launches (serving: vectors for different
// operators).  k_mx_slice_G_many slices the columns of every G_d (warp per column;
// CTA x holds columns 4 (x - blk0) .. of the descriptor whose range holds it), then
// k_mx_apply_many runs the 64 x 64 tiles of every V_d = T_d G_d.
template <int S>
__global__ void __launch_bounds__(128) k_mx_slice_G_many(const MxApplyDesc *__restrict__ ds, int nd) {
    int lo = 0, hi = nd - 1;
    const int x = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ds[mid].blk0 <= x) lo = mid;
        else hi = mid - 1;
    }
    const MxApplyDesc D = ds[lo];
    const int j = (x - D.blk0) * 4 + (threadIdx.x >> 5);
    if (j >= D.B) return;
    auto get = [&](int kk) -> float2 { return df_from_d(D.G[(size_t)j * D.N + kk]); };
    warp_slice_row<S>(get, D.N, D.kpad, D.gdig, D.gplane, j, D.gex);
}

template <int S>
__global__ void __launch_bounds__(PIPE_THREADS) k_mx_apply_many(const MxApplyDesc *__restrict__ ds, int nd) {
    extern __shared__ __align__(16) unsigned char smem_raw[];  // pipe_smem_bytes(S)
    int lo = 0, hi = nd - 1;
    const int x = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ds[mid].tile0 <= x) lo = mid;
        else hi = mid - 1;
    }
    const MxApplyDesc D = ds[lo];
    const int t = x - D.tile0, ti = (D.N + 63) / 64;
    const int i0 = (t % ti) * 64, j0 = (t / ti) * 64, N = D.N, B = D.B;
    double *V = D.V;
    digit_gemm_pipe<S>(D.tdig, (int64_t)N * D.kpad, D.kpad, i0, N, D.tex, D.gdig, D.gplane, D.kpad, j0, B, D.gex, N,
                       (__nv_bfloat16 *)smem_raw, [&](const int *r, const int *cl, const float2 *v, bool first) {
#pragma unroll
                           for (int q = 0; q < 4; ++q) {
                               const int i = i0 + r[q], j = j0 + cl[q];
                               if (i >= N || j >= B) continue;
                               double *o = V + (size_t)j * N + i;
                               *o = first ? df_to_d(v[q]) : *o + df_to_d(v[q]);
                           }
                       });
}

// ----------------------------------------------------------------------------- launchers

#define MX_SPLIT_DISPATCH(split, CALL) \
    do {                                \
        switch (split) {                \
        case 3: { constexpr int SS = 3; CALL; } break; \
        case 4: { constexpr int SS = 4; CALL; } break; \
        case 6: { constexpr int SS = 6; CALL; } break; \
        default: { constexpr int SS = 5; CALL; } break; \
        }                               \
    } while (0)

cudaError_t mx_convert(const double *x, float2 *y, int64_t n, cudaStream_t s, KTimer &kt) {
    int bx = (int)std::min<int64_t>((n + 255) / 256, 8192);
    if (bx < 1) bx = 1;
    kt.begin(GM_K_ASSEMBLE, 0.0, s);
    k_mx_d2df<<<bx, 256, 0, s>>>(x, y, n);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t mx_merge_assemble(const MergeDesc *md, int nm, const int *tab, const float2 *in, float2 *ws,
                              int64_t max_elems, const double *b, const double *c, const double *d, int n,
                              cudaStream_t s, KTimer &kt) {
    int bx = (int)((max_elems + 1023) / 1024);
    if (bx < 1) bx = 1;
    if (bx > 4096) bx = 4096;
    kt.begin(GM_K_ASSEMBLE, 0.0, s);
    k_mx_merge_assemble<<<dim3(bx, nm), 256, 0, s>>>(md, tab, in, ws, b, c, d, n);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t mx_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                        float2 *ws, int nb, int split, MxScratch &scr, Status *st, int stage, cudaStream_t s,
                        KTimer &kt) {
    const int smem_limit = 200 * 1024;
    const int nsys = (int)h_sys.size();
    // the default 48 KiB limit counts the kernel's static shared memory (about 5 KiB)
    // too, so the limit is raised whatever the panel size
    {
        cudaError_t e = cudaFuncSetAttribute(k_mx_gj_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k < max_m; k += nb) {
        int rows = max_m - k;
        int nbe = nb < rows ? nb : rows;
        double fl_panel = 0, fl_piv = 0, fl_upd = 0;
        for (const SysDesc &S : h_sys) {
            if (k >= S.m) continue;
            double e = std::min(nb, S.m - k), r = S.m - k, cols = S.ncol - k - e;
            fl_panel += r * e * e;
            fl_piv += 2.0 * e * e * cols;
            fl_upd += 2.0 * (S.m - e) * e * cols;
        }
        size_t smem = (size_t)rows * nbe * sizeof(float);
        if (smem > (size_t)smem_limit) return cudaErrorInvalidValue;
        kt.begin(GM_K_PANEL, fl_panel, s);
        k_mx_gj_panel<<<nsys, MX_PANEL_THREADS, smem, s>>>(d_sys, ws, k, nb, scr.perm, scr.perm_n, scr.a11inv, st,
                                                           stage);
        kt.end(s);
        const int cols = max_ncol - k;
        const int cb = (cols + 127) / 128, rb = (max_m + 127) / 128;
        kt.begin(GM_K_PIVROWS, fl_piv, s);
        MX_SPLIT_DISPATCH(split, (k_mx_gj_prep<SS><<<dim3(cb + rb, nsys), 128, 0, s>>>(
                                     d_sys, ws, k, nb, cb, scr.perm, scr.perm_n, scr.a11inv, scr.fdig, scr.fplane,
                                     scr.fex, scr.rdig, scr.rplane, scr.rex)));
        kt.end(s);
        dim3 g3((max_m + 63) / 64, (cols + 63) / 64, nsys);
        kt.begin(GM_K_GJUPDATE, fl_upd, s);
        MX_SPLIT_DISPATCH(split, (k_mx_gj_update<SS><<<g3, 128, 0, s>>>(d_sys, ws, k, nb, scr.fdig, scr.fplane,
                                                                          scr.fex, scr.rdig, scr.rplane, scr.rex)));
        kt.end(s);
    }
    return cudaGetLastError();
}

cudaError_t mx_merge_update(const MergeDesc *md, const std::vector<MergeDesc> &h_md, const int *tab,
                            const float2 *in, const float2 *ws, float2 *out, int max_rp, int split,
                            __nv_bfloat16 *ydig, int *yex, __nv_bfloat16 *xdig, int *xex, int64_t plane,
                            const double *b, const double *c, const double *d, int n, Status *st, cudaStream_t s,
                            KTimer &kt, int wait_limit, int tc_min_k) {
    double fl = 0;
    for (const MergeDesc &M : h_md) fl += 2.0 * (double)M.rp * M.rp * M.sp;
    const int nm = (int)h_md.size();
    const int rb = (max_rp + 3) / 4;
    int max_kpad = 0;
    for (const MergeDesc &M : h_md) max_kpad = std::max(max_kpad, M.kpad);
    const bool tc = max_kpad >= tc_min_k;  // the tcgen05 kernel reads tile-ordered digit planes
    kt.begin(GM_K_MERGEUPDATE, fl, s);
    MX_SPLIT_DISPATCH(split, (k_mx_merge_slice<SS><<<dim3(2 * rb, nm), 128, 0, s>>>(md, tab, in, ws, rb, ydig, yex,
                                                                                      xdig, xex, plane, tc ? 1 : 0)));
    cudaError_t e = cudaSuccess;
    if (!tc) {  // short K: the pipeline's fill and drain would dominate
        const dim3 g64((max_rp + 63) / 64, (max_rp + 63) / 64, nm);
        MX_SPLIT_DISPATCH(split, (e = cudaFuncSetAttribute(k_mx_merge_update<SS>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)pipe_smem_bytes(SS))));
        if (e != cudaSuccess) return e;
        MX_SPLIT_DISPATCH(split, (k_mx_merge_update<SS><<<g64, PIPE_THREADS, pipe_smem_bytes(SS), s>>>(
                                     md, tab, in, out, ydig, yex, xdig, xex, plane, b, c, d, n)));
        kt.end(s);
        return cudaGetLastError();
    }
    // tcgen05 tiles of 128 x 64 (tensor memory: 512 columns per CTA, one CTA per SM by
    // shared memory, so the allocation never waits)
    dim3 g((max_rp + MT_ROWS - 1) / MT_ROWS, (max_rp + MT_COLS - 1) / MT_COLS, nm);
    MX_SPLIT_DISPATCH(split, (e = cudaFuncSetAttribute(k_mx_merge_update_tc<SS>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)mx_merge_tc_smem(SS))));
    if (e != cudaSuccess) return e;
    MX_SPLIT_DISPATCH(split, (k_mx_merge_update_tc<SS><<<g, PIPE_THREADS, mx_merge_tc_smem(SS), s>>>(
                                 md, tab, in, out, ydig, yex, xdig, xex, plane, b, c, d, st, wait_limit)));
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t mx_root_assemble(const float2 *S, int r, int n, float2 *ws, const double *b, const double *c,
                             const double *d, cudaStream_t s, KTimer &kt) {
    int64_t tot = (int64_t)r * (r + 4 * n);
    int bx = (int)std::min<int64_t>((tot + 1023) / 1024, 8192);
    kt.begin(GM_K_ASSEMBLE, 0.0, s);
    k_mx_root_assemble<<<bx, 256, 0, s>>>(S, r, n, ws, b, c, d);
    kt.end(s);
    return cudaGetLastError();
}

int mx_kpad(int N) { return (N + 15) / 16 * 16; }

cudaError_t mx_root_finalize(const float2 *ws, int r, int n, double *T, float2 *Tdf, __nv_bfloat16 *tdig, int *tex,
                             int split, Status *st, int stage, cudaStream_t s, KTimer &kt) {
    const int N = 4 * n, kpad = mx_kpad(N);
    int64_t tot = (int64_t)N * N;
    int bx = (int)std::min<int64_t>((tot + 1023) / 1024, 8192);
    kt.begin(GM_K_ROOT, 0.0, s);
    k_mx_root_finalize<<<bx, 256, 0, s>>>(ws, r, n, T, Tdf, st, stage);
    MX_SPLIT_DISPATCH(split, (k_mx_slice_T<SS><<<(N + 3) / 4, 128, 0, s>>>(Tdf, N, kpad, tdig, (int64_t)N * kpad,
                                                                           tex)));
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t mx_apply_many(std::vector<MxApplyDesc> &h, MxApplyDesc *d, int split, cudaStream_t s) {
    int tiles = 0, blks = 0;
    for (MxApplyDesc &q : h) {
        q.tile0 = tiles;
        q.blk0 = blks;
        tiles += ((q.N + 63) / 64) * ((q.B + 63) / 64);
        blks += (q.B + 3) / 4;
    }
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(MxApplyDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const int nd = (int)h.size();
    MX_SPLIT_DISPATCH(split, (k_mx_slice_G_many<SS><<<blks, 128, 0, s>>>(d, nd)));
    MX_SPLIT_DISPATCH(split, (e = cudaFuncSetAttribute(k_mx_apply_many<SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)pipe_smem_bytes(SS))));
    if (e != cudaSuccess) return e;
    MX_SPLIT_DISPATCH(split, (k_mx_apply_many<SS><<<tiles, PIPE_THREADS, pipe_smem_bytes(SS), s>>>(d, nd)));
    return cudaGetLastError();
}

cudaError_t mx_apply(const __nv_bfloat16 *tdig, const int *tex, const double *G, __nv_bfloat16 *gdig, int *gex,
                     double *V, int N, int B, int split, cudaStream_t s) {
    const int kpad = mx_kpad(N);
    MX_SPLIT_DISPATCH(split, (k_mx_slice_G<SS><<<(B + 3) / 4, 128, 0, s>>>(G, N, B, kpad, gdig, (int64_t)B * kpad,
                                                                           gex)));
    dim3 g((N + 63) / 64, (B + 63) / 64);
    cudaError_t e = cudaSuccess;
    MX_SPLIT_DISPATCH(split, (e = cudaFuncSetAttribute(k_mx_apply<SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)pipe_smem_bytes(SS))));
    if (e != cudaSuccess) return e;
    MX_SPLIT_DISPATCH(split, (k_mx_apply<SS><<<g, PIPE_THREADS, pipe_smem_bytes(SS), s>>>(
                                 tdig, tex, (int64_t)N * kpad, gdig, gex, (int64_t)B * kpad, kpad, V, N, B)));
    return cudaGetLastError();
}

}  // namespace gm
