// FP64 kernels of the dense build and solve.
//
//   k_leaf          leaf Schur complement, eq. def_schur_nd (Section 3.1), banded A_ii
//                   (Section 3.4 cost remark)
//   k_merge_*       pairwise merge, eq. S_fromtwo_nd (Section 3.2)
//   k_gj_*          batched blocked Gauss-Jordan elimination with partial pivoting that
//                   turns [M | Z] into [* | M^{-1} Z] (the interface solve of a merge and
//                   the root inversion, Section 3.3 step 4)
//   k_root_*        root: T = (I - P S^{-1} B)/h
//   k_apply         solve stage: V = T G (Section 1.1)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gm_internal.h"
#include "kernels.h"
#include "smem_limit.h"

namespace gm {

// ----------------------------------------------------------------------------- stencil

// Weight of the equation at global node g on its neighbour in direction dir (Section 6).
// With c == nullptr, b is a table of five weights per node (centre, E, W, N, S; the
// conductance networks of Section 6.1).
__device__ __forceinline__ double stencil_w(const double *__restrict__ b, const double *__restrict__ c,
                                            const double *__restrict__ d, double ih, int g, int dir) {
    if (!c) return b[5 * (int64_t)g + dir];
    // ih = 1/h = n+1 exactly: no FP64 division (a long instruction sequence on GB300)
    const double ih2 = ih * ih;
    switch (dir) {
    case DIR_C: return 4.0 * ih2 + d[g];
    case DIR_E: return -ih2 + b[g] * ih;
    case DIR_W: return -ih2 - b[g] * ih;
    case DIR_N: return -ih2 + c[g] * ih;
    default: return -ih2 - c[g] * ih;
    }
}

__device__ __forceinline__ void ring_node(int a, int b, int p, int &i, int &j) {
    if (p <= a - 1) { i = p; j = 0; }
    else if (p <= a + b - 2) { i = a - 1; j = p - a + 1; }
    else if (p <= 2 * a + b - 3) { i = 2 * a + b - 3 - p; j = b - 1; }
    else { i = 0; j = 2 * a + 2 * b - 4 - p; }
}

__device__ __forceinline__ int ring_pos_d(int a, int b, int i, int j) {
    if (j == 0) return i;
    if (i == a - 1) return a - 1 + j;
    if (j == b - 1) return (a - 1) + (b - 1) + (a - 1 - i);
    if (i == 0) return 2 * (a - 1) + (b - 1) + (b - 1 - j);
    return -1;
}

__device__ __forceinline__ void record_pivot(Status *st, double piv, int stage) {
    double ap = fabs(piv);
    if (!(ap > 0.0) || !isfinite(ap)) {
        if (atomicCAS(&st->code, 0, GM_ESINGULAR) == 0) st->where = stage;
        return;
    }
    atomicMin(&st->min_piv, (unsigned long long)__double_as_longlong(ap));
}

// ----------------------------------------------------------------------------- leaf

// One CTA per leaf.  Shared memory: band of A_ii (ni x W), solves X (ni x nq), index
// maps.  A_ii is eliminated by banded Gaussian elimination with partial pivoting; the
// unit right-hand sides are the interior nodes next to the ring, because A_ib and
// A_bi couple each non-corner ring node to exactly one interior node.
__global__ void __launch_bounds__(LEAF_THREADS)
k_leaf(const LeafDesc *__restrict__ leaves, const double *__restrict__ bf0, const double *__restrict__ cf0,
       const double *__restrict__ df0, double *__restrict__ out, Status *st, int stage) {
    extern __shared__ double sm[];
    const LeafDesc Ld = leaves[blockIdx.x];
    const int n = Ld.n;
    const double *bf = bf0 + Ld.coef, *cf = cf0 + Ld.coef, *df = df0 + Ld.coef;
    const int a = Ld.a, bb = Ld.b;
    const int ia = a - 2, ib = bb - 2;
    const int ni = (ia > 0 && ib > 0) ? ia * ib : 0;
    const int r = 2 * a + 2 * bb - 4;
    const int KL = ia, UW = 2 * ia, W = 3 * ia + 1;
    const double ih = n + 1.0;  // 1/h
    const int tid = threadIdx.x, nt = blockDim.x;

    // inner-ring interior nodes (those with a ring neighbour)
    int nq = 0;
    if (ni > 0) nq = (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
    double *band = sm;                   // ni * W
    double *X = band + (size_t)ni * W;   // ni * nq
    int *piv = (int *)(X + (size_t)ni * nq);
    int *inner_id = piv + ni;            // ni
    int *inner_q = inner_id + ni;        // nq

    auto gnode = [&](int ii, int jj) { return (Ld.x0 + 1 + ii) + n * (Ld.y0 + 1 + jj); };

    if (ni > 0) {
        for (int e = tid; e < ni * W; e += nt) band[e] = 0.0;
        __syncthreads();
        for (int q = tid; q < ni; q += nt) {
            int ii = q % ia, jj = q / ia;
            int g = gnode(ii, jj);
            double *row = band + (size_t)q * W + KL - q;  // row[col] for col in band
            row[q] = stencil_w(bf, cf, df, ih, g, DIR_C);
            if (ii + 1 < ia) row[q + 1] = stencil_w(bf, cf, df, ih, g, DIR_E);
            if (ii > 0) row[q - 1] = stencil_w(bf, cf, df, ih, g, DIR_W);
            if (jj + 1 < ib) row[q + ia] = stencil_w(bf, cf, df, ih, g, DIR_N);
            if (jj > 0) row[q - ia] = stencil_w(bf, cf, df, ih, g, DIR_S);
            bool edge = (ii == 0 || ii == ia - 1 || jj == 0 || jj == ib - 1);
            inner_id[q] = edge ? 1 : -1;
        }
        __syncthreads();
        if (tid == 0) {
            int c = 0;
            for (int q = 0; q < ni; ++q)
                if (inner_id[q] >= 0) { inner_id[q] = c; inner_q[c] = q; ++c; }
        }
        __syncthreads();
        // banded LU with partial pivoting (row interchanges limited to the band)
        const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
        __shared__ int s_p;
        // Until the first row interchange every row r reaches at most column r + KL, so
        // the elimination (and later the backward sweep) can stop there: diagonally
        // dominant leaves never pay for the 2 KL fill that pivoting could create.
        bool swapped = false;
        for (int k = 0; k < ni; ++k) {
            const int last = min(k + KL, ni - 1);
            if (tid < 32) {
                int rr = k + tid;
                double v = (rr <= last) ? fabs(band[(size_t)rr * W + KL + k - rr]) : -1.0;
                int idx = rr;
                for (int o = 16; o > 0; o >>= 1) {
                    double v2 = __shfl_down_sync(0xffffffffu, v, o);
                    int i2 = __shfl_down_sync(0xffffffffu, idx, o);
                    if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
                }
                // a NaN column leaves no candidate: keep the diagonal (every access in bounds)
                if (tid == 0) {
                    if (idx < k || idx > last) idx = k;
                    s_p = idx;
                    piv[k] = idx;
                }
            }
            __syncthreads();
            const int p = s_p;
            swapped = swapped || p != k;
            const int cend = min(k + (swapped ? UW : KL), ni - 1);
            if (p != k) {
                for (int cc = k + tid; cc <= cend; cc += nt) {
                    double *x = &band[(size_t)k * W + KL + cc - k];
                    double *y = &band[(size_t)p * W + KL + cc - p];
                    double t = *x; *x = *y; *y = t;
                }
            }
            __syncthreads();
            const double pv = band[(size_t)k * W + KL];
            if (tid == 0) record_pivot(st + Ld.prob, pv, stage);
            if (tid < last - k) {  // only the threads that scale divide (FP64 division is long)
                const int rr = k + 1 + tid;
                band[(size_t)rr * W + KL + k - rr] /= pv;
            }
            __syncthreads();
            const int nr = last - k, ncn = cend - k;
            for (int e = tid; e < nr * ncn; e += nt) {
                int rr = k + 1 + e / ncn, cc = k + 1 + e % ncn;
                band[(size_t)rr * W + KL + cc - rr] -= band[(size_t)rr * W + KL + k - rr] * band[(size_t)k * W + KL + cc - k];
            }
            __syncthreads();
        }
        const int UWe = swapped ? UW : KL;  // upper bandwidth of U
        double *idg = (double *)(inner_q + nq + (nq & 1));  // reciprocals of U's diagonal
        for (int k = tid; k < ni; k += nt) idg[k] = 1.0 / band[(size_t)k * W + KL];
        // one unit right-hand side per inner-ring node (column t of X)
        for (int e = tid; e < ni * nq; e += nt) X[e] = 0.0;
        __syncthreads();
        for (int t = tid; t < nq; t += nt) X[(size_t)inner_q[t] * nq + t] = 1.0;
        __syncthreads();
        // forward and backward sweeps: the right-hand sides are independent, so each warp
        // owns up to 8 of them (lanes: 8 columns x 4 row slices) and syncs only itself
        {
            const int cpw = (nq + nwarp - 1) / nwarp;  // columns per warp (<= 8: nq <= 64)
            const int cl = lane & 7, rs = lane >> 3;
            const int t = warp * cpw + cl;
            const bool on = cl < cpw && t < nq;
            for (int k = 0; k < ni; ++k) {  // forward: interchange, then eliminate below row k
                const int p = piv[k];
                if (on && rs == 0 && p != k) {
                    const double a0 = X[(size_t)k * nq + t];
                    X[(size_t)k * nq + t] = X[(size_t)p * nq + t];
                    X[(size_t)p * nq + t] = a0;
                }
                __syncwarp();
                if (on) {
                    const int last = min(k + KL, ni - 1);
                    const double xk = X[(size_t)k * nq + t];
                    for (int rr = k + 1 + rs; rr <= last; rr += 4)
                        X[(size_t)rr * nq + t] -= band[(size_t)rr * W + KL + k - rr] * xk;
                }
                __syncwarp();
            }
            for (int k = ni - 1; k >= 0; --k) {  // backward: divide row k, eliminate above it
                if (on && rs == 0) X[(size_t)k * nq + t] *= idg[k];
                __syncwarp();
                if (on) {
                    const int r0 = max(0, k - UWe);
                    const double xk = X[(size_t)k * nq + t];
                    for (int rr = r0 + rs; rr < k; rr += 4) X[(size_t)rr * nq + t] -= band[(size_t)rr * W + KL + k - rr] * xk;
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
    // S[l, m] = A_bb[l, m] - w(l -> ql) (A_ii^{-1})[ql, qm] w(qm -> m)
    double *S = out + Ld.off;
    for (int e = tid; e < r * r; e += nt) {
        int l = e % r, m = e / r;  // column-major: row l, column m
        int il, jl, im, jm;
        ring_node(a, bb, l, il, jl);
        ring_node(a, bb, m, im, jm);
        int gl = (Ld.x0 + il) + n * (Ld.y0 + jl);
        double v = 0.0;
        int dx = im - il, dy = jm - jl;
        if (dx == 0 && dy == 0) v = stencil_w(bf, cf, df, ih, gl, DIR_C);
        else if (dx == 1 && dy == 0) v = stencil_w(bf, cf, df, ih, gl, DIR_E);
        else if (dx == -1 && dy == 0) v = stencil_w(bf, cf, df, ih, gl, DIR_W);
        else if (dx == 0 && dy == 1) v = stencil_w(bf, cf, df, ih, gl, DIR_N);
        else if (dx == 0 && dy == -1) v = stencil_w(bf, cf, df, ih, gl, DIR_S);
        if (ni > 0) {
            // interior neighbour of a non-corner ring node, and the direction to it
            auto inner = [&](int i, int j, int &ii, int &jj, int &dir) -> bool {
                if (j == 0 && i > 0 && i < a - 1) { ii = i - 1; jj = 0; dir = DIR_N; return true; }
                if (j == bb - 1 && i > 0 && i < a - 1) { ii = i - 1; jj = ib - 1; dir = DIR_S; return true; }
                if (i == 0 && j > 0 && j < bb - 1) { ii = 0; jj = j - 1; dir = DIR_E; return true; }
                if (i == a - 1 && j > 0 && j < bb - 1) { ii = ia - 1; jj = j - 1; dir = DIR_W; return true; }
                return false;
            };
            int il2, jl2, dl, im2, jm2, dm;
            if (inner(il, jl, il2, jl2, dl) && inner(im, jm, im2, jm2, dm)) {
                int ql = il2 + ia * jl2, qm = im2 + ia * jm2;
                int gm_ = gnode(im2, jm2);
                // direction from the interior node qm back to ring node m is opposite of dm
                int back = (dm == DIR_N) ? DIR_S : (dm == DIR_S) ? DIR_N : (dm == DIR_E) ? DIR_W : DIR_E;
                double wl = stencil_w(bf, cf, df, ih, gl, dl);
                double wm = stencil_w(bf, cf, df, ih, gm_, back);
                v -= wl * X[(size_t)ql * nq + inner_id[qm]] * wm;
            }
        }
        S[e] = v;
    }
}

size_t leaf_smem_bytes(int a, int b) {
    int ia = a - 2, ib = b - 2;
    int ni = (ia > 0 && ib > 0) ? ia * ib : 0;
    int nq = 0;
    if (ni > 0) nq = (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
    int W = 3 * (ia > 0 ? ia : 0) + 1;
    return (size_t)ni * W * 8 + (size_t)ni * nq * 8 + (size_t)(2 * ni + nq + 1) * 4 + (size_t)ni * 8 + 16;
}

// ----------------------------------------------------------------------------- Gauss-Jordan sweep

// Panel factorisation: LU with partial pivoting of rows k..m-1 of columns k..k+nbe-1.
// One CTA per system; the panel lives in shared memory (SMEM) or stays in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(GJ_PANEL_THREADS)
k_gj_panel(const SysDesc *__restrict__ sys, double *__restrict__ ws, int k, int nb, int *__restrict__ piv,
           int piv_ld, Status *st, int stage) {
    extern __shared__ double smp[];
    __shared__ double s_val[32];
    __shared__ int s_idx[32];
    const SysDesc S = sys[blockIdx.x];
    const int m = S.m;
    if (k >= m) return;
    const int nbe = min(nb, m - k), rows = m - k;
    double *A = ws + S.off;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    double *P;
    int ldp;
    if (SMEM) {
        P = smp;
        ldp = rows;
        for (int e = tid; e < rows * nbe; e += nt) {
            int rr = e % rows, c = e / rows;
            P[(size_t)c * ldp + rr] = A[(size_t)(k + c) * m + k + rr];
        }
        __syncthreads();
    } else {
        P = A + (size_t)k * m + k;
        ldp = m;
    }
    for (int t = 0; t < nbe; ++t) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int rr = t + tid; rr < rows; rr += nt) {
            double v = fabs(P[(size_t)t * ldp + rr]);
            if (v > best) { best = v; bi = rr; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double v2 = __shfl_down_sync(0xffffffffu, best, o);
            int i2 = __shfl_down_sync(0xffffffffu, bi, o);
            if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (wid == 0) {
            best = lane < nw ? s_val[lane] : -1.0;
            bi = lane < nw ? s_idx[lane] : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                double v2 = __shfl_down_sync(0xffffffffu, best, o);
                int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
            }
            if (lane == 0) {
                // an all-NaN column (after an earlier zero pivot) leaves no candidate:
                // keep the diagonal row so every access stays inside the panel
                if (bi < t || bi >= rows) bi = t;
                s_idx[0] = bi;
                piv[(size_t)blockIdx.x * piv_ld + k + t] = k + bi;
            }
        }
        __syncthreads();
        const int pr = s_idx[0];
        if (pr != t) {
            for (int c = tid; c < nbe; c += nt) {
                double x = P[(size_t)c * ldp + t];
                P[(size_t)c * ldp + t] = P[(size_t)c * ldp + pr];
                P[(size_t)c * ldp + pr] = x;
            }
        }
        __syncthreads();
        const double pv = P[(size_t)t * ldp + t];
        if (tid == 0) record_pivot(st + S.prob, pv, stage);
        const double inv = 1.0 / pv;
        for (int rr = t + 1 + tid; rr < rows; rr += nt) {
            double l = P[(size_t)t * ldp + rr] * inv;
            P[(size_t)t * ldp + rr] = l;
            for (int c = t + 1; c < nbe; ++c) P[(size_t)c * ldp + rr] -= l * P[(size_t)c * ldp + t];
        }
        __syncthreads();
    }
    if (SMEM) {
        for (int e = tid; e < rows * nbe; e += nt) {
            int rr = e % rows, c = e / rows;
            A[(size_t)(k + c) * m + k + rr] = P[(size_t)c * ldp + rr];
        }
    }
}

// Pivot rows: apply the panel's row interchanges to every column right of the panel,
// then U12 = L11^{-1} A12 (kept aside for the rows below) and R = U11^{-1} U12 (written
// into the pivot rows, used for the rows above).  One thread per column.
__global__ void __launch_bounds__(128)
k_gj_pivrows(const SysDesc *__restrict__ sys, double *__restrict__ ws, int k, int nb,
             const int *__restrict__ piv, int piv_ld, double *__restrict__ u12, int64_t u12_stride) {
    __shared__ double LU[GJ_MAX_NB][GJ_MAX_NB];
    __shared__ int pv[GJ_MAX_NB];
    const SysDesc S = sys[blockIdx.y];
    const int m = S.m;
    if (k >= m) return;
    const int nbe = min(nb, m - k);
    double *A = ws + S.off;
    for (int e = threadIdx.x; e < nbe * nbe; e += blockDim.x) {
        int i = e % nbe, j = e / nbe;
        LU[i][j] = A[(size_t)(k + j) * m + k + i];
    }
    for (int e = threadIdx.x; e < nbe; e += blockDim.x) pv[e] = piv[(size_t)blockIdx.y * piv_ld + k + e];
    __syncthreads();
    const int j = k + nbe + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S.ncol) return;
    double *col = A + (size_t)j * m;
    double v[GJ_MAX_NB];
#pragma unroll
    for (int t = 0; t < GJ_MAX_NB; ++t) {
        if (t < nbe) {
            int p = pv[t];
            double x = col[k + t];
            if (p != k + t) { double y = col[p]; col[p] = x; x = y; }
            v[t] = x;
        }
    }
    double *U = u12 + (size_t)blockIdx.y * u12_stride;
#pragma unroll
    for (int t = 0; t < GJ_MAX_NB; ++t) {
        if (t < nbe) {
            double s = v[t];
#pragma unroll
            for (int q = 0; q < GJ_MAX_NB; ++q)
                if (q < t) s -= LU[t][q] * v[q];
            v[t] = s;
            U[(size_t)t * S.ncol + j] = s;
        }
    }
#pragma unroll
    for (int t = GJ_MAX_NB - 1; t >= 0; --t) {
        if (t < nbe) {
            double s = v[t];
#pragma unroll
            for (int q = 0; q < GJ_MAX_NB; ++q)
                if (q > t && q < nbe) s -= LU[t][q] * v[q];
            v[t] = s / LU[t][t];
            col[k + t] = v[t];
        }
    }
}

// Rank-nbe update of every non-pivot row: rows below use L21 * U12, rows above use
// A01 * R.  64 x 64 tile per CTA, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256)
k_gj_update(const SysDesc *__restrict__ sys, double *__restrict__ ws, int k, int nb,
            const double *__restrict__ u12, int64_t u12_stride) {
    __shared__ double F[GJ_MAX_NB][64];
    __shared__ double Gu[GJ_MAX_NB][64];
    __shared__ double Gr[GJ_MAX_NB][64];
    const SysDesc S = sys[blockIdx.z];
    const int m = S.m;
    if (k >= m) return;
    const int nbe = min(nb, m - k);
    const int i0 = blockIdx.x * 64, j0 = k + nbe + blockIdx.y * 64;
    if (i0 >= m || j0 >= S.ncol) return;
    double *A = ws + S.off;
    const double *U = u12 + (size_t)blockIdx.z * u12_stride;
    const int tid = threadIdx.x;
    for (int e = tid; e < nbe * 64; e += 256) {
        int t = e / 64, x = e % 64;
        int i = i0 + x, j = j0 + x;
        F[t][x] = (i < m) ? A[(size_t)(k + t) * m + i] : 0.0;
        Gu[t][x] = (j < S.ncol) ? U[(size_t)t * S.ncol + j] : 0.0;
        Gr[t][x] = (j < S.ncol) ? A[(size_t)j * m + k + t] : 0.0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int t = 0; t < nbe; ++t) {
        double f[4], gu[4], gr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            f[q] = F[t][tx + 16 * q];
            gu[q] = Gu[t][ty + 16 * q];
            gr[q] = Gr[t][ty + 16 * q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool below = (i0 + tx + 16 * q) >= k + nbe;
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] += f[q] * (below ? gu[p] : gr[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int j = j0 + ty + 16 * p;
        if (j >= S.ncol) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = i0 + tx + 16 * q;
            if (i >= m || (i >= k && i < k + nbe)) continue;
            A[(size_t)j * m + i] -= acc[q][p];
        }
    }
}

// ----------------------------------------------------------------------------- merges

struct MergeTab {
    const int *p3, *p4, *g3, *g4, *p1, *q1, *p2, *q2, *x12;
};
__device__ __forceinline__ MergeTab merge_tab(const MergeDesc &M, const int *tab) {
    const int *t = tab + M.tab;
    MergeTab T;
    T.p3 = t; T.p4 = t + M.sp; T.g3 = t + 2 * M.sp; T.g4 = t + 3 * M.sp;
    T.p1 = t + 4 * M.sp; T.q1 = T.p1 + M.n1; T.p2 = T.q1 + M.n1; T.q2 = T.p2 + M.n2;
    T.x12 = T.q2 + M.n2;
    return T;
}

// [M | Z] with M = [S33 A34; A43 S44], Z = [S31 0; 0 S42] (eq. S_fromtwo_nd; the
// five-point stencil makes A14, A23, A32, A41 vanish).
__global__ void __launch_bounds__(256)
k_merge_assemble(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const double *__restrict__ in,
                 double *__restrict__ ws, const double *__restrict__ bf, const double *__restrict__ cf,
                 const double *__restrict__ df, int n) {
    const MergeDesc M = md[blockIdx.y];
    const MergeTab T = merge_tab(M, tab);
    const int sp = M.sp, mm = 2 * sp, ncol = mm + M.rp;
    const int64_t tot = (int64_t)mm * ncol;
    const double *S1 = in + M.s1, *S2 = in + M.s2;
    double *A = ws + M.ws;
    const double ih = M.n + 1.0;  // 1/h of the merge's problem
    const int d34 = M.orient ? DIR_N : DIR_E, d43 = M.orient ? DIR_S : DIR_W;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int t = (int)(e % mm), c = (int)(e / mm);
        double v = 0.0;
        if (c < mm) {
            if (t < sp && c < sp) v = S1[T.p3[t] + (int64_t)M.r1 * T.p3[c]];
            else if (t >= sp && c >= sp) v = S2[T.p4[t - sp] + (int64_t)M.r2 * T.p4[c - sp]];
            else if (t < sp) v = (c - sp == t) ? stencil_w(bf, cf, df, ih, T.g3[t], d34) : 0.0;
            else v = (c == t - sp) ? stencil_w(bf, cf, df, ih, T.g4[t - sp], d43) : 0.0;
        } else {
            int cc = c - mm;
            if (cc < M.n1) v = (t < sp) ? S1[T.p3[t] + (int64_t)M.r1 * T.p1[cc]] : 0.0;
            else v = (t >= sp) ? S2[T.p4[t - sp] + (int64_t)M.r2 * T.p2[cc - M.n1]] : 0.0;
        }
        A[e] = v;
    }
}

// The parent's Schur complement of a 64 x 64 tile: C - acc with C = [S11 A12; A21 S22]
// (A12, A21 the two corner couplings across the shared edge), scattered into the
// parent's ring order.  Thread (tx, ty) holds rows a0 + tx + 16 q, columns c0 + ty + 16 p.
__device__ __forceinline__ void merge_store(const MergeDesc &M, const MergeTab &T, const double *__restrict__ S1,
                                            const double *__restrict__ S2, double *__restrict__ out,
                                            const double (&acc)[4][4], int a0, int c0, int tx, int ty,
                                            const double *__restrict__ bf, const double *__restrict__ cf,
                                            const double *__restrict__ df) {
    const int rp = M.rp, n1 = M.n1;
    const double ih = M.n + 1.0;  // 1/h of the merge's problem
    const int d12 = M.orient ? DIR_N : DIR_E, d21 = M.orient ? DIR_S : DIR_W;
    double *O = out + M.out;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int cc = c0 + ty + 16 * p;
        if (cc >= rp) continue;
        int qc = cc < n1 ? T.q1[cc] : T.q2[cc - n1];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int aa = a0 + tx + 16 * q;
            if (aa >= rp) continue;
            int qa = aa < n1 ? T.q1[aa] : T.q2[aa - n1];
            double cval = 0.0;
            if (aa < n1 && cc < n1) cval = S1[T.p1[aa] + (int64_t)M.r1 * T.p1[cc]];
            else if (aa >= n1 && cc >= n1) cval = S2[T.p2[aa - n1] + (int64_t)M.r2 * T.p2[cc - n1]];
            else {
                for (int e = 0; e < 2; ++e) {
                    const int *x = T.x12 + 4 * e;
                    if (aa < n1 && aa == x[0] && cc - n1 == x[1]) cval = stencil_w(bf, cf, df, ih, x[2], d12);
                    if (aa >= n1 && aa - n1 == x[1] && cc == x[0]) cval = stencil_w(bf, cf, df, ih, x[3], d21);
                }
            }
            O[qa + (int64_t)rp * qc] = cval - acc[q][p];
        }
    }
}

// S_parent = [S11 A12; A21 S22] - [S13 0; 0 S24] X, scattered into the parent's ring
// order.  X = M^{-1} Z is the right block of the workspace after the sweep.
__global__ void __launch_bounds__(256)
k_merge_update(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const double *__restrict__ in,
               const double *__restrict__ ws, double *__restrict__ out, const double *__restrict__ bf,
               const double *__restrict__ cf, const double *__restrict__ df, int n) {
    __shared__ double Y[64][17];
    __shared__ double X1[16][64];
    __shared__ double X2[16][64];
    const MergeDesc M = md[blockIdx.z];
    const int rp = M.rp;
    const int a0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
    if (a0 >= rp || c0 >= rp) return;
    const MergeTab T = merge_tab(M, tab);
    const int sp = M.sp, mm = 2 * sp, n1 = M.n1;
    const double *S1 = in + M.s1, *S2 = in + M.s2;
    const double *Xw = ws + M.ws + (size_t)mm * mm;  // X: mm x rp, ld = mm
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int t0 = 0; t0 < sp; t0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            int x = e % 64, t = e / 64;  // Y: row a0+x, interface column t0+t
            int aa = a0 + x, tt = t0 + t;
            double y = 0.0;
            if (aa < rp && tt < sp)
                y = (aa < n1) ? S1[T.p1[aa] + (int64_t)M.r1 * T.p3[tt]] : S2[T.p2[aa - n1] + (int64_t)M.r2 * T.p4[tt]];
            Y[x][t] = y;
            int cc = c0 + x;
            X1[t][x] = (cc < rp && tt < sp) ? Xw[(size_t)cc * mm + tt] : 0.0;
            X2[t][x] = (cc < rp && tt < sp) ? Xw[(size_t)cc * mm + sp + tt] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 16; ++t) {
            double y[4], x1[4], x2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                y[q] = Y[tx + 16 * q][t];
                x1[q] = X1[t][ty + 16 * q];
                x2[q] = X2[t][ty + 16 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool top = (a0 + tx + 16 * q) < n1;
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += y[q] * (top ? x1[p] : x2[p]);
            }
        }
        __syncthreads();
    }
    merge_store(M, T, S1, S2, out, acc, a0, c0, tx, ty, bf, cf, df);
}

// Step 2 of the accelerated merge (Section 5, eq. matmult): the product of the update in
// factored form, [L13 W13; L24 W24] with W13 = R13 X3, W24 = R24 X4 (S13 ~ L13 R13 and
// S24 ~ L24 R24 at the compression tolerance), then the same assembly and ring scatter
// as k_merge_update (Step 3, the parent formed densely).  One merge per launch.
__global__ void __launch_bounds__(256)
k_merge_update_lr(const MergeDesc *__restrict__ md, const int *__restrict__ tab, const double *__restrict__ in,
                  const LrUpdate lr, double *__restrict__ out, const double *__restrict__ bf,
                  const double *__restrict__ cf, const double *__restrict__ df) {
    __shared__ double Y[64][17];
    __shared__ double X1[16][64];
    __shared__ double X2[16][64];
    const MergeDesc M = *md;
    const int rp = M.rp;
    const int a0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
    if (a0 >= rp || c0 >= rp) return;
    const MergeTab T = merge_tab(M, tab);
    const int n1 = M.n1, K = max(lr.k13, lr.k24);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int t0 = 0; t0 < K; t0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            const int x = e % 64, t = e / 64, aa = a0 + x, tt = t0 + t, cc = c0 + x;
            double y = 0.0;
            if (aa < n1) {
                if (tt < lr.k13) y = lr.L13[aa + (size_t)tt * n1];
            } else if (aa < rp && tt < lr.k24) {
                y = lr.L24[(aa - n1) + (size_t)tt * (rp - n1)];
            }
            Y[x][t] = y;
            X1[t][x] = (cc < rp && tt < lr.k13) ? lr.W13[tt + (size_t)cc * lr.k13] : 0.0;
            X2[t][x] = (cc < rp && tt < lr.k24) ? lr.W24[tt + (size_t)cc * lr.k24] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int t = 0; t < 16; ++t) {
            double y[4], x1[4], x2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                y[q] = Y[tx + 16 * q][t];
                x1[q] = X1[t][ty + 16 * q];
                x2[q] = X2[t][ty + 16 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool top = (a0 + tx + 16 * q) < n1;
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += y[q] * (top ? x1[p] : x2[p]);
            }
        }
        __syncthreads();
    }
    merge_store(M, T, in + M.s1, in + M.s2, out, acc, a0, c0, tx, ty, bf, cf, df);
}

// ----------------------------------------------------------------------------- root

// Ghost k -> (flat index of its unknown neighbour, direction from that neighbour to k).
__device__ __forceinline__ void ghost_nb(int n, int k, int &g, int &dir) {
    int side = k / n, t = k % n;
    if (side == 0) { g = t; dir = DIR_S; }
    else if (side == 1) { g = (n - 1) + n * t; dir = DIR_E; }
    else if (side == 2) { g = (n - 1 - t) + n * (n - 1); dir = DIR_N; }
    else { g = n * (n - 1 - t); dir = DIR_W; }
}

// Root ring position of ghost k's neighbour: (k - floor(k/n)) mod (4n - 4).
__device__ __forceinline__ int ghost_ring(int n, int k) {
    int r = 4 * n - 4;
    int p = k - k / n;
    return p >= r ? p - r : p;
}

// [S_root | B], B(ring(k), k) = -w_k: the ghost couplings moved to the right-hand side.
__global__ void k_root_assemble(const double *__restrict__ S, int r, int n, double *__restrict__ ws,
                                const double *__restrict__ bf, const double *__restrict__ cf,
                                const double *__restrict__ df) {
    const int64_t tot = (int64_t)r * (r + 4 * n);
    const double ih = n + 1.0;  // 1/h
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int row = (int)(e % r), c = (int)(e / r);
        double v;
        if (c < r) v = S[e];
        else {
            int k = c - r, g, dir;
            ghost_nb(n, k, g, dir);
            v = (row == ghost_ring(n, k)) ? -stencil_w(bf, cf, df, ih, g, dir) : 0.0;
        }
        ws[e] = v;
    }
}

// T[k, k'] = (delta_kk' - X[ring(k), k'])/h, X = S_root^{-1} B.
__global__ void k_root_finalize(const double *__restrict__ ws, int r, int n, double *__restrict__ T) {
    const int nb4 = 4 * n;
    const int64_t tot = (int64_t)nb4 * nb4;
    const double ih = n + 1.0;  // 1/h
    const double *X = ws + (size_t)r * r;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(e % nb4), kp = (int)(e / nb4);
        double x = X[(size_t)kp * r + ghost_ring(n, k)];
        T[e] = ((k == kp ? 1.0 : 0.0) - x) * ih;
    }
}

// ----------------------------------------------------------------------------- apply

// One 64 x 64 tile of V = T G: T is N x N, G and V are N x B, all column-major.
__device__ __forceinline__ void apply_tile(const double *__restrict__ T, const double *__restrict__ G,
                                           double *__restrict__ V, int N, int B, int i0, int j0) {
    __shared__ double At[16][65];
    __shared__ double Bt[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < N; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            int x = e % 64, t = e / 64;
            int i = i0 + x, kk = k0 + t;
            At[t][x] = (i < N && kk < N) ? T[(size_t)kk * N + i] : 0.0;
            int kk2 = k0 + (e % 16), j = j0 + e / 16;
            Bt[e % 16][e / 16] = (kk2 < N && j < B) ? G[(size_t)j * N + kk2] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = At[t][tx + 16 * q]; b[q] = Bt[t][ty + 16 * q]; }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += a[q] * b[p];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        int j = j0 + ty + 16 * p;
        if (j >= B) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int i = i0 + tx + 16 * q;
            if (i < N) V[(size_t)j * N + i] = acc[q][p];
        }
    }
}

// V = T G, 64 x 64 tile per CTA.
__global__ void __launch_bounds__(256)
k_apply(const double *__restrict__ T, const double *__restrict__ G, double *__restrict__ V, int N, int B) {
    apply_tile(T, G, V, N, B, blockIdx.x * 64, blockIdx.y * 64);
}

// V_d = T_d G_d for several operators in one launch: CTA x takes tile x - tile0 of the
// descriptor whose range holds it (descriptors sorted by tile0, found by bisection).
__global__ void __launch_bounds__(256) k_apply_many(const ApplyDesc *__restrict__ ds, int nd) {
    int lo = 0, hi = nd - 1;
    const int x = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ds[mid].tile0 <= x) lo = mid;
        else hi = mid - 1;
    }
    const ApplyDesc D = ds[lo];
    const int t = x - D.tile0, ti = (D.N + 63) / 64;
    apply_tile(D.T, D.G, D.V, D.N, D.B, (t % ti) * 64, (t / ti) * 64);
}

// ----------------------------------------------------------------------------- launchers

cudaError_t launch_leaf(const LeafDesc *d_leaves, const std::vector<LeafDesc> &h_leaves, int max_a, int max_b,
                        const double *b, const double *c, const double *d, double *out, Status *st, int stage,
                        cudaStream_t s, KTimer &kt) {
    size_t smem = leaf_smem_bytes(max_a, max_b);
    // always raise the limit: the default 48 KiB counts static shared memory too
    cudaError_t e = raise_smem_limit((const void *)k_leaf, smem);
    if (e != cudaSuccess) return e;
    // banded LU ~ 4 ni ia^2, one forward + backward solve per inner-ring node ~ 6 ni ia
    double fl = 0.0;
    for (const LeafDesc &L : h_leaves) {
        double ia = L.a - 2, ib = L.b - 2;
        if (ia <= 0 || ib <= 0) continue;
        double ni = ia * ib, nq = (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
        fl += 4.0 * ni * ia * ia + 6.0 * nq * ni * ia;
    }
    kt.begin(GM_K_LEAF, fl, s);
    k_leaf<<<(int)h_leaves.size(), LEAF_THREADS, smem, s>>>(d_leaves, b, c, d, out, st, stage);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t launch_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                            double *ws, int nb, int *piv, int piv_ld, double *u12, int64_t u12_stride, Status *st,
                            int stage, cudaStream_t s, KTimer &kt) {
    const int smem_limit = 200 * 1024;
    const int nsys = (int)h_sys.size();
    // the panel of the first step is the largest; the default 48 KiB limit counts the
    // kernel's static shared memory too, so the limit is raised whatever the size
    {
        cudaError_t e = cudaFuncSetAttribute(k_gj_panel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
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
            // algorithmic (LU) count: rows below the panel over every remaining column, rows
            // above it over the right-hand sides only (the rest is the Gauss-Jordan sweep's
            // extra m^3/3 over an LU with back substitution)
            fl_upd += 2.0 * e * ((S.m - k - e) * cols + (double)k * (S.ncol - S.m));
        }
        size_t smem = (size_t)rows * nbe * sizeof(double);
        kt.begin(GM_K_PANEL, fl_panel, s);
        if (smem <= (size_t)smem_limit) {
            k_gj_panel<true><<<nsys, GJ_PANEL_THREADS, smem, s>>>(d_sys, ws, k, nb, piv, piv_ld, st, stage);
        } else {
            k_gj_panel<false><<<nsys, GJ_PANEL_THREADS, 0, s>>>(d_sys, ws, k, nb, piv, piv_ld, st, stage);
        }
        kt.end(s);
        // columns right of the panel; systems with a narrower last panel need up to nb more
        int cols = max_ncol - k;
        dim3 g2((cols + 127) / 128, nsys);
        kt.begin(GM_K_PIVROWS, fl_piv, s);
        k_gj_pivrows<<<g2, 128, 0, s>>>(d_sys, ws, k, nb, piv, piv_ld, u12, u12_stride);
        kt.end(s);
        dim3 g3((max_m + 63) / 64, (cols + 63) / 64, nsys);
        kt.begin(GM_K_GJUPDATE, fl_upd, s);
        k_gj_update<<<g3, 256, 0, s>>>(d_sys, ws, k, nb, u12, u12_stride);
        kt.end(s);
    }
    return cudaGetLastError();
}

cudaError_t launch_merge_assemble(const MergeDesc *md, int nm, const int *tab, const double *in, double *ws,
                                  int64_t max_elems, const double *b, const double *c, const double *d, int n,
                                  cudaStream_t s, KTimer &kt) {
    int bx = (int)((max_elems + 1023) / 1024);
    if (bx < 1) bx = 1;
    if (bx > 4096) bx = 4096;
    kt.begin(GM_K_ASSEMBLE, 0.0, s);
    k_merge_assemble<<<dim3(bx, nm), 256, 0, s>>>(md, tab, in, ws, b, c, d, n);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t launch_merge_update_lr(const MergeDesc *md, const MergeDesc &h_md, const int *tab, const double *in,
                                   const LrUpdate &lr, double *out, const double *b, const double *c, const double *d,
                                   cudaStream_t s, KTimer &kt) {
    const int rp = h_md.rp, K = std::max(lr.k13, lr.k24);
    dim3 g((rp + 63) / 64, (rp + 63) / 64, 1);
    kt.begin(GM_K_MERGEUPDATE, 2.0 * (double)rp * rp * K, s);
    k_merge_update_lr<<<g, 256, 0, s>>>(md, tab, in, lr, out, b, c, d);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t launch_merge_update(const MergeDesc *md, const std::vector<MergeDesc> &h_md, const int *tab,
                                const double *in, const double *ws, double *out, int max_rp, const double *b,
                                const double *c, const double *d, int n, cudaStream_t s, KTimer &kt) {
    double fl = 0;
    for (const MergeDesc &M : h_md) fl += 2.0 * (double)M.rp * M.rp * M.sp;
    dim3 g((max_rp + 63) / 64, (max_rp + 63) / 64, (int)h_md.size());
    kt.begin(GM_K_MERGEUPDATE, fl, s);
    k_merge_update<<<g, 256, 0, s>>>(md, tab, in, ws, out, b, c, d, n);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t launch_root_assemble(const double *S, int r, int n, double *ws, const double *b, const double *c,
                                 const double *d, cudaStream_t s, KTimer &kt) {
    int64_t tot = (int64_t)r * (r + 4 * n);
    int bx = (int)((tot + 1023) / 1024);
    if (bx > 8192) bx = 8192;
    kt.begin(GM_K_ASSEMBLE, 0.0, s);
    k_root_assemble<<<bx, 256, 0, s>>>(S, r, n, ws, b, c, d);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t launch_root_finalize(const double *ws, int r, int n, double *T, cudaStream_t s, KTimer &kt) {
    int64_t tot = (int64_t)16 * n * n;
    int bx = (int)((tot + 1023) / 1024);
    if (bx > 8192) bx = 8192;
    kt.begin(GM_K_ROOT, 0.0, s);
    k_root_finalize<<<bx, 256, 0, s>>>(ws, r, n, T);
    kt.end(s);
    return cudaGetLastError();
}

cudaError_t launch_apply_many(std::vector<ApplyDesc> &h, ApplyDesc *d, cudaStream_t s) {
    int tiles = 0;
    for (ApplyDesc &q : h) {
        q.tile0 = tiles;
        tiles += ((q.N + 63) / 64) * ((q.B + 63) / 64);
    }
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(ApplyDesc), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_apply_many<<<tiles, 256, 0, s>>>(d, (int)h.size());
    return cudaGetLastError();
}

cudaError_t launch_apply(const double *T, const double *G, double *V, int N, int B, cudaStream_t s) {
    dim3 g((N + 63) / 64, (B + 63) / 64);
    k_apply<<<g, 256, 0, s>>>(T, G, V, N, B);
    return cudaGetLastError();
}

}  // namespace gm
