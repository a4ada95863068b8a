// Kernels of the body-load build (Section 6.3): the leaves' load maps, the load columns of
// every merge, the root's load operator F and its apply.  The interface systems, leaf
// Schur complements, merge updates and root of the same build run on the FP64 kernels of
// kernels_fp64.cu; these kernels only add the load columns around them.  All loops are
// grid-stride loops bounded by the element counts of their descriptors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "loads.h"

namespace gm {

namespace {

// Weight of the equation at global node g on its neighbour in direction dir (the
// Section 6 stencil, as the FP64 kernels evaluate it: ih = 1/h = n + 1 exactly; with
// c == nullptr, b is a table of five weights per node, as for a conductance network).
__device__ __forceinline__ double ld_stencil(const double *__restrict__ b, const double *__restrict__ c,
                                             const double *__restrict__ d, double ih, int g, int dir) {
    if (!c) return b[5 * (int64_t)g + dir];
    const double ih2 = ih * ih;
    switch (dir) {
    case DIR_C: return 4.0 * ih2 + d[g];
    case DIR_E: return -ih2 + b[g] * ih;
    case DIR_W: return -ih2 - b[g] * ih;
    case DIR_N: return -ih2 + c[g] * ih;
    default: return -ih2 - c[g] * ih;
    }
}

// Local (i, j) of ring position p of an a x b box (counter-clockwise from the SW corner).
__device__ __forceinline__ void ld_ring_node(int a, int b, int p, int &i, int &j) {
    if (p <= a - 1) { i = p; j = 0; }
    else if (p <= a + b - 2) { i = a - 1; j = p - a + 1; }
    else if (p <= 2 * a + b - 3) { i = 2 * a + b - 3 - p; j = b - 1; }
    else { i = 0; j = 2 * a + 2 * b - 4 - p; }
}

// Root ring position of ghost k's neighbour (ghosts counter-clockwise from the SW corner).
__device__ __forceinline__ int ld_ghost_ring(int n, int k) {
    const int r = 4 * n - 4;
    const int p = k - k / n;
    return p >= r ? p - r : p;
}

// A merge's index table (layout in gm_internal.h).
struct LdTab {
    const int *p3, *p4, *p1, *q1, *p2, *q2;
};
__device__ __forceinline__ LdTab ld_tab(const MergeDesc &M, const int *__restrict__ tab) {
    const int *t = tab + M.tab;
    LdTab T;
    T.p3 = t;
    T.p4 = t + M.sp;
    T.p1 = t + 4 * M.sp;
    T.q1 = T.p1 + M.n1;
    T.p2 = T.q1 + M.n1;
    T.q2 = T.p2 + M.n2;
    return T;
}

// The four neighbour directions q = 0..3: east, west, north, south.
__device__ __forceinline__ int ld_dir(int q) { return q == 0 ? DIR_E : q == 1 ? DIR_W : q == 2 ? DIR_N : DIR_S; }
__device__ __forceinline__ int ld_di(int q) { return q == 0 ? 1 : q == 1 ? -1 : 0; }
__device__ __forceinline__ int ld_dj(int q) { return q == 2 ? 1 : q == 3 ? -1 : 0; }

}  // namespace

// [A_ii | E_i] of a leaf with loads: A_ii from the stencil on the interior nodes (index
// (i-1) + (a-2)(j-1) for local (i, j)), E_i the unit columns of its interior body nodes.
__global__ void __launch_bounds__(256)
k_leaf_load_assemble(const LeafLoadDesc *__restrict__ D, const int *__restrict__ nodes, double *__restrict__ ws,
                     const double *__restrict__ bf, const double *__restrict__ cf, const double *__restrict__ df) {
    const LeafLoadDesc L = D[blockIdx.y];
    if (L.sys < 0) return;
    const int ni = L.ni, ia = L.a - 2, n = L.n;
    const int64_t tot = (int64_t)ni * (ni + L.m);
    const double ih = n + 1.0;
    double *W = ws + L.sys;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(e % ni), col = (int)(e / ni);
        const int i = 1 + p % ia, j = 1 + p / ia;
        const int g = (L.x0 + i) + n * (L.y0 + j);
        double v = 0.0;
        if (col < ni) {
            const int iq = 1 + col % ia, jq = 1 + col / ia;
            if (col == p) {
                v = ld_stencil(bf, cf, df, ih, g, DIR_C);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (iq == i + ld_di(q) && jq == j + ld_dj(q)) v = ld_stencil(bf, cf, df, ih, g, ld_dir(q));
            }
        } else {
            v = nodes[L.col0 + (col - ni)] == g ? 1.0 : 0.0;
        }
        W[e] = v;
    }
}

// L = E_b - A_bi X with X = A_ii^{-1} E_i the right block of the swept system: each ring
// node couples to its interior neighbours (at most one for a box of edge >= 3).
__global__ void __launch_bounds__(256)
k_leaf_load_finalize(const LeafLoadDesc *__restrict__ D, const int *__restrict__ nodes, const double *__restrict__ ws,
                     double *__restrict__ larena, const double *__restrict__ bf, const double *__restrict__ cf,
                     const double *__restrict__ df) {
    const LeafLoadDesc L = D[blockIdx.y];
    const int a = L.a, b = L.b, n = L.n, ni = L.ni, ia = a - 2;
    const int r = 2 * a + 2 * b - 4;
    const int64_t tot = (int64_t)r * L.m;
    const double ih = n + 1.0;
    const double *X = L.sys >= 0 ? ws + L.sys + (int64_t)ni * ni : nullptr;
    double *out = larena + L.lout;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int rb = (int)(e % r), col = (int)(e / r);
        int i, j;
        ld_ring_node(a, b, rb, i, j);
        const int g = (L.x0 + i) + n * (L.y0 + j);
        double v = nodes[L.col0 + col] == g ? 1.0 : 0.0;
        if (X) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i2 = i + ld_di(q), j2 = j + ld_dj(q);
                if (i2 >= 1 && i2 <= a - 2 && j2 >= 1 && j2 <= b - 2)
                    v -= ld_stencil(bf, cf, df, ih, g, ld_dir(q)) * X[(i2 - 1) + ia * (j2 - 1) + (int64_t)ni * col];
            }
        }
        out[e] = v;
    }
}

// The load columns of a merge's system, after [M | Z]: [L1(P3) 0; 0 L2(P4)].
__global__ void __launch_bounds__(256)
k_merge_load_assemble(const MergeDesc *__restrict__ md, const MergeLoadDesc *__restrict__ ld,
                      const int *__restrict__ tab, const double *__restrict__ larena, double *__restrict__ ws) {
    const MergeDesc M = md[blockIdx.y];
    const MergeLoadDesc D = ld[blockIdx.y];
    const int sp = M.sp, mm = 2 * sp, mL = D.m1 + D.m2;
    if (mL == 0 || mm == 0) return;
    const LdTab T = ld_tab(M, tab);
    double *Z = ws + M.ws + (int64_t)mm * (mm + M.rp);
    const int64_t tot = (int64_t)mm * mL;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e % mm), col = (int)(e / mm);
        double v = 0.0;
        if (t < sp && col < D.m1) v = larena[D.l1 + T.p3[t] + (int64_t)M.r1 * col];
        else if (t >= sp && col >= D.m1) v = larena[D.l2 + T.p4[t - sp] + (int64_t)M.r2 * (col - D.m1)];
        Z[e] = v;
    }
}

// The parent's load map: [L1(P1) 0; 0 L2(P2)] - [S13 0; 0 S24] X_L, rows in the parent's
// ring order, X_L the load columns of the swept system (rows 0..sp-1 for child 1's side,
// sp..2sp-1 for child 2's).
__global__ void __launch_bounds__(256)
k_merge_load_update(const MergeDesc *__restrict__ md, const MergeLoadDesc *__restrict__ ld,
                    const int *__restrict__ tab, const double *__restrict__ in, const double *__restrict__ ws,
                    double *__restrict__ larena) {
    const MergeDesc M = md[blockIdx.y];
    const MergeLoadDesc D = ld[blockIdx.y];
    const int sp = M.sp, mm = 2 * sp, mL = D.m1 + D.m2, rp = M.rp, n1 = M.n1;
    if (mL == 0) return;
    const LdTab T = ld_tab(M, tab);
    const double *S1 = in + M.s1, *S2 = in + M.s2;
    const double *XL = ws + M.ws + (int64_t)mm * (mm + rp);
    double *out = larena + D.lout;
    const int64_t tot = (int64_t)rp * mL;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e % rp), col = (int)(e / rp);
        double g = 0.0, acc = 0.0;
        int qa;
        if (a < n1) {
            if (col < D.m1) g = larena[D.l1 + T.p1[a] + (int64_t)M.r1 * col];
            for (int t = 0; t < sp; ++t) acc += S1[T.p1[a] + (int64_t)M.r1 * T.p3[t]] * XL[t + (int64_t)mm * col];
            qa = T.q1[a];
        } else {
            const int a2 = a - n1;
            if (col >= D.m1) g = larena[D.l2 + T.p2[a2] + (int64_t)M.r2 * (col - D.m1)];
            for (int t = 0; t < sp; ++t)
                acc += S2[T.p2[a2] + (int64_t)M.r2 * T.p4[t]] * XL[sp + t + (int64_t)mm * col];
            qa = T.q2[a2];
        }
        out[qa + (int64_t)rp * col] = g - acc;
    }
}

// F[k, order[c]] = -X_L[ring(k), c] / h: the ghost data of the root solve with the loads
// of tree column c (the datum of the Section 6 problem is the plain one-sided flux).
__global__ void __launch_bounds__(256)
k_load_finalize(const double *__restrict__ xl, int r, int n, int m, const int *__restrict__ order,
                double *__restrict__ F) {
    const int nb4 = 4 * n;
    const int64_t tot = (int64_t)nb4 * m;
    const double ih = n + 1.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % nb4), col = (int)(e / nb4);
        F[k + (int64_t)nb4 * order[col]] = -xl[ld_ghost_ring(n, k) + (int64_t)r * col] * ih;
    }
}

// V += F Fl: F is N x m, Fl m x B, V N x B, all column-major.  16 x 16 output tiles.
__global__ void __launch_bounds__(256)
k_apply_add(const double *__restrict__ F, const double *__restrict__ Fl, double *__restrict__ V, int N, int m, int B) {
    __shared__ double Ft[16][17], Lt[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.x * 16 + tx, col = blockIdx.y * 16 + ty;
    double acc = 0.0;
    for (int k0 = 0; k0 < m; k0 += 16) {
        const int fr = blockIdx.x * 16 + tx, fk = k0 + ty;
        Ft[ty][tx] = (fr < N && fk < m) ? F[fr + (int64_t)N * fk] : 0.0;
        const int lk = k0 + tx, lc = blockIdx.y * 16 + ty;
        Lt[ty][tx] = (lk < m && lc < B) ? Fl[lk + (int64_t)m * lc] : 0.0;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) acc += Ft[q][tx] * Lt[ty][q];
        __syncthreads();
    }
    if (row < N && col < B) V[row + (int64_t)N * col] += acc;
}

// ----------------------------------------------------------------------------- launchers

namespace {
int grid_for(int64_t elems, int cap) {
    int64_t g = (elems + 255) / 256;
    if (g < 1) g = 1;
    return (int)std::min<int64_t>(g, cap);
}
}  // namespace

cudaError_t launch_leaf_load_assemble(const LeafLoadDesc *d, int nl, const int *nodes, double *ws, int max_elems,
                                      const double *b, const double *c, const double *dd, cudaStream_t s) {
    if (nl == 0) return cudaSuccess;
    k_leaf_load_assemble<<<dim3(grid_for(max_elems, 1024), nl), 256, 0, s>>>(d, nodes, ws, b, c, dd);
    return cudaGetLastError();
}

cudaError_t launch_leaf_load_finalize(const LeafLoadDesc *d, int nl, const int *nodes, const double *ws,
                                      double *larena, int max_rm, const double *b, const double *c,
                                      const double *dd, cudaStream_t s) {
    if (nl == 0) return cudaSuccess;
    k_leaf_load_finalize<<<dim3(grid_for(max_rm, 1024), nl), 256, 0, s>>>(d, nodes, ws, larena, b, c, dd);
    return cudaGetLastError();
}

cudaError_t launch_merge_load_assemble(const MergeDesc *md, const MergeLoadDesc *ld, int nm, const int *tab,
                                       const double *larena, double *ws, int64_t max_elems, cudaStream_t s) {
    if (nm == 0) return cudaSuccess;
    k_merge_load_assemble<<<dim3(grid_for(max_elems, 1024), nm), 256, 0, s>>>(md, ld, tab, larena, ws);
    return cudaGetLastError();
}

cudaError_t launch_merge_load_update(const MergeDesc *md, const MergeLoadDesc *ld, int nm, const int *tab,
                                     const double *in, const double *ws, double *larena, int64_t max_elems,
                                     cudaStream_t s) {
    if (nm == 0) return cudaSuccess;
    k_merge_load_update<<<dim3(grid_for(max_elems, 1024), nm), 256, 0, s>>>(md, ld, tab, in, ws, larena);
    return cudaGetLastError();
}

cudaError_t launch_load_finalize(const double *xl, int r, int n, int m, const int *order, double *F, cudaStream_t s) {
    k_load_finalize<<<grid_for((int64_t)4 * n * m, 8192), 256, 0, s>>>(xl, r, n, m, order, F);
    return cudaGetLastError();
}

cudaError_t launch_apply_add(const double *F, const double *Fl, double *V, int N, int m, int B, cudaStream_t s) {
    if (m == 0 || B == 0) return cudaSuccess;
    dim3 g((N + 15) / 16, (B + 15) / 16);
    k_apply_add<<<g, 256, 0, s>>>(F, Fl, V, N, m, B);
    return cudaGetLastError();
}

}  // namespace gm
