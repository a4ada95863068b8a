// HBS root (Sections 4 and 5): the root Schur complement S (r x r) compressed to HBS
// factors {D, U, V, B} over a binary tree of its ring, inverted by Algorithm 1, and
// applied by Algorithm 2 in the solve stage: dudn = (g - P S^{-1} B g)/h.
//
// GB300 design.  Every dense step is a batch of small FP64 products described by a
// descriptor array (one launch per level and kind); the bases come from randomized
// samples Y = S Omega, Z = S^T Psi (one large product each), so that no node ever
// touches its wide off-diagonal block row: a node's sample is its rows of Y minus the
// part of S inside the node (leaves) or its children's reduced samples minus the
// sibling coupling (parents).  Each sample (at most 192 x 128) is reduced by a
// column-pivoted Gram-Schmidt QR in shared memory (one CTA per node), truncated at the
// first |R_jj| <= tol |R_11|.  The dense inversions of Algorithm 1 reuse the batched
// Gauss-Jordan sweep on [M | I].  Ranks are read back once per level.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "hbs.h"
#include "network.h"
#include "smem_limit.h"

namespace gm {

namespace {

// ----------------------------------------------------------------------------- kernels

// Standard normal samples: SplitMix64 (Steele, Lea & Flood 2014) counter stream, uniform
// doubles from the top 53 bits, Box-Muller on pairs (u1 mapped to (0, 1]).
__device__ __forceinline__ unsigned long long splitmix(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_hbs_normals(double *__restrict__ out, int64_t count, unsigned long long seed) {
    const int64_t pairs = (count + 1) / 2;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pairs; p += (int64_t)gridDim.x * blockDim.x) {
        const double u1 = 1.0 - (double)(splitmix(seed, 2 * p) >> 11) * (1.0 / 9007199254740992.0);
        const double u2 = (double)(splitmix(seed, 2 * p + 1) >> 11) * (1.0 / 9007199254740992.0);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        out[2 * p] = rad * cs;
        if (2 * p + 1 < count) out[2 * p + 1] = rad * sn;
    }
}

// C (m x n) = alpha op(A) op(B) + beta C, FP64, column-major; op(X) = X or X^T.
struct GemmDesc {
    const double *A, *B;
    double *C;
    int m, n, k, lda, ldb, ldc, ta, tb;
    double alpha, beta;
};

// One 64 x 64 tile of one descriptor per CTA (blockIdx.z = descriptor).  Operand tiles
// are staged through shared memory with the contiguous dimension fastest across
// threads, whichever the transposition.
__global__ void __launch_bounds__(256) k_hgemm(const GemmDesc *__restrict__ ds) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const GemmDesc D = ds[blockIdx.z];
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    if (i0 >= D.m || j0 >= D.n) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < D.k; k0 += 16) {
        for (int e = tid; e < 16 * 64; e += 256) {
            int x, t;
            if (D.ta) { t = e & 15; x = e >> 4; } else { x = e & 63; t = e >> 6; }
            const int i = i0 + x, kk = k0 + t;
            double a = 0.0;
            if (i < D.m && kk < D.k) a = D.ta ? D.A[kk + (size_t)i * D.lda] : D.A[i + (size_t)kk * D.lda];
            As[t][x] = a;
            if (D.tb) { x = e & 63; t = e >> 6; } else { t = e & 15; x = e >> 4; }
            const int j = j0 + x, k2 = k0 + t;
            double b = 0.0;
            if (j < D.n && k2 < D.k) b = D.tb ? D.B[j + (size_t)k2 * D.ldb] : D.B[k2 + (size_t)j * D.ldb];
            Bs[t][x] = b;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[t][tx + 16 * q];
                b[q] = Bs[t][ty + 16 * q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] = fma(a[q], b[p], acc[q][p]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int j = j0 + ty + 16 * p;
        if (j >= D.n) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + tx + 16 * q;
            if (i >= D.m) continue;
            double *c = D.C + i + (size_t)j * D.ldc;
            *c = D.beta == 0.0 ? D.alpha * acc[q][p] : fma(D.beta, *c, D.alpha * acc[q][p]);
        }
    }
}

// dst (rows x cols) = src, or the identity (src == nullptr, mode 1), or zero (mode 2).
struct CopyDesc {
    const double *src;
    double *dst;
    int rows, cols, lds, ldd, mode, pad;
};

__global__ void k_hbs_copy(const CopyDesc *__restrict__ ds) {
    const CopyDesc D = ds[blockIdx.y];
    const int64_t tot = (int64_t)D.rows * D.cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % D.rows), j = (int)(e / D.rows);
        double v;
        if (D.mode == 0) v = D.src[i + (size_t)j * D.lds];
        else if (D.mode == 1) v = (i == j) ? 1.0 : 0.0;
        else v = 0.0;
        D.dst[i + (size_t)j * D.ldd] = v;
    }
}

// Basis of the column space of A (p x l) by Gram-Schmidt with column pivoting: at step j
// the remaining column of largest norm is re-orthogonalised against Q(:, 0..j-1),
// normalised into Q(:, j) and removed from every other remaining column.
// out[0] = first j with |R_jj| <= tol |R_11| (or the steps taken), out[1] = columns of
// Q produced.  The sweep stops at a numerically zero column, after kmax columns, or
// `margin` columns past the truncation point (the partner basis of the same node may
// truncate a little later; one rank serves both).
//
// Two kernels: a single CTA with A in shared memory for small samples (p <= QR_MAXP,
// l <= HBS_SAMPLES), and a thread-block cluster for large ones (k_hbs_pqr_cl).
constexpr int QR_MAXP = 192;

struct QrDesc {
    const double *A;  // p x l sample (read only)
    double *Q;        // p x (columns produced), ld ldq
    int *out;         // [truncation point, columns produced]
    double *W;        // p x l work copy (cluster kernel only)
    int p, l, lda, ldq;
};

__device__ __forceinline__ double warp_sum_d(double s) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void __launch_bounds__(256) k_hbs_pqr(const QrDesc *__restrict__ ds, double tol, int kmax, int margin) {
    extern __shared__ double sA[];  // [l][p] column-major
    __shared__ double nrm[HBS_SAMPLES];
    __shared__ double qv[QR_MAXP];
    __shared__ double coef[QR_MAXP];
    __shared__ unsigned char used[HBS_SAMPLES];
    __shared__ int s_piv;
    __shared__ double s_r, s_r1;
    const QrDesc D = ds[blockIdx.x];
    const int p = D.p, l = D.l, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int e = tid; e < p * l; e += blockDim.x) {
        const int i = e % p, j = e / p;
        sA[(size_t)j * p + i] = D.A[i + (size_t)j * D.lda];
    }
    for (int j = tid; j < l; j += blockDim.x) used[j] = 0;
    __syncthreads();
    // the columns' squared norms; each step below refreshes them while it removes q
    for (int c = warp; c < l; c += nw) {
        double s = 0.0;
        for (int i = lane; i < p; i += 32) s = fma(sA[(size_t)c * p + i], sA[(size_t)c * p + i], s);
        s = warp_sum_d(s);
        if (lane == 0) nrm[c] = s;
    }
    __syncthreads();
    int ktr = -1, kval = 0;
    const int steps = min(kmax, min(p, l));
    for (int j = 0; j < steps; ++j) {
        if (warp == 0) {  // the unused column of largest norm, the lowest on ties
            double bv = -1.0;
            int bc = 0x7fffffff;
            for (int c = lane; c < l; c += 32)
                if (!used[c] && nrm[c] > bv) {
                    bv = nrm[c];
                    bc = c;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
                if (ov > bv || (ov == bv && oc < bc)) {
                    bv = ov;
                    bc = oc;
                }
            }
            if (lane == 0) {
                s_piv = bv >= 0.0 ? bc : -1;
                s_r = bv > 0.0 ? sqrt(bv) : 0.0;
                if (j == 0) s_r1 = s_r;
            }
        }
        __syncthreads();
        const int pv = s_piv;
        const double rjj = s_r, r11 = s_r1;
        if (ktr < 0 && !(rjj > tol * r11)) ktr = j;
        if (pv < 0 || !(rjj > 1e-15 * r11) || !(r11 > 0.0) || (ktr >= 0 && j >= ktr + margin)) break;
        for (int i = tid; i < p; i += blockDim.x) qv[i] = sA[(size_t)pv * p + i];
        __syncthreads();
        // the pivot column has had every earlier q removed (below); one more pass
        // q -= Q (Q^T q) restores the orthogonality the roundings took
        for (int c = warp; c < j; c += nw) {
            double s = 0.0;
            for (int i = lane; i < p; i += 32) s = fma(D.Q[i + (size_t)c * D.ldq], qv[i], s);
            s = warp_sum_d(s);
            if (lane == 0) coef[c] = s;
        }
        __syncthreads();
        double ss = 0.0;
        for (int i = tid; i < p; i += blockDim.x) {
            double v = qv[i];
            for (int c = 0; c < j; ++c) v = fma(-coef[c], D.Q[i + (size_t)c * D.ldq], v);
            qv[i] = v;
            ss = fma(v, v, ss);
        }
        ss = warp_sum_d(ss);
        if (lane == 0) coef[QR_MAXP - 1 - warp] = ss;  // per-warp partial sums (j < QR_MAXP - nw)
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += coef[QR_MAXP - 1 - w];
            s_r = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
            used[pv] = 1;
        }
        __syncthreads();
        const double inv = s_r;
        for (int i = tid; i < p; i += blockDim.x) {
            qv[i] *= inv;
            D.Q[i + (size_t)j * D.ldq] = qv[i];
        }
        __syncthreads();
        // remove q from every remaining column and refresh its norm
        for (int c = warp; c < l; c += nw) {
            if (used[c]) continue;
            double s = 0.0;
            for (int i = lane; i < p; i += 32) s = fma(qv[i], sA[(size_t)c * p + i], s);
            s = warp_sum_d(s);
            double nn = 0.0;
            for (int i = lane; i < p; i += 32) {
                const double v = fma(-s, qv[i], sA[(size_t)c * p + i]);
                sA[(size_t)c * p + i] = v;
                nn = fma(v, v, nn);
            }
            nn = warp_sum_d(nn);
            if (lane == 0) nrm[c] = nn;
        }
        __syncthreads();
        kval = j + 1;
    }
    if (tid == 0) {
        D.out[0] = ktr < 0 ? kval : ktr;
        D.out[1] = kval;
    }
}

// The same factorisation on a thread-block cluster: the CTAs of a cluster share one
// sample, CTA c owning the columns g = c + cs i (cs = cluster size).  The columns live in
// a global work copy W (L2-resident), read and written through L2 only, so that every
// CTA sees the others' latest values.  One step:
//   1. each CTA offers its unused column of largest norm; after a cluster barrier every
//      CTA reads all offers from distributed shared memory and takes the same pivot
//      (largest norm, lowest column on ties);
//   2. each CTA forms the part of Q (Q^T a) that falls on its own columns of Q and
//      publishes it in its shared memory; after a second barrier every CTA subtracts all
//      parts in the same order and normalises, so all hold the same q bit for bit; the
//      pivot's owner stores it as Q(:, j);
//   3. each CTA removes q from its unused columns and refreshes their norms.
// Offers and parts alternate between two buffers, so two barriers per step suffice; a
// final barrier keeps every CTA's shared memory alive until the others are done with it.
constexpr int QRC_THREADS = 512;
constexpr int QRC_LOC = HBS_MAX_SAMPLES / 8;  // columns per CTA at the smallest cluster (8)
constexpr int QRC_MAXP = 8000;                // rows: 3 p doubles of dynamic shared memory
constexpr int QRC_MAXP_G = 1 << 20;           // rows with the vectors in global memory instead

// gscr == nullptr: the CTA's q vector and its two part buffers live in dynamic shared
// memory (p <= QRC_MAXP) and the others' parts are read through distributed shared
// memory; otherwise CTA b keeps them in global memory at gscr + b * 3 * pstride (taller
// samples, up to QRC_MAXP_G rows) and reads the others' parts from there.
__global__ void __launch_bounds__(QRC_THREADS) k_hbs_pqr_cl(const QrDesc *__restrict__ ds, double tol, int kmax,
                                                           int margin, double *__restrict__ gscr, int pstride) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int cs = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    const QrDesc D = ds[blockIdx.x / cs];
    extern __shared__ double smx[];  // qv[p], part[2][p] (without gscr)
    __shared__ double nrm[QRC_LOC];
    __shared__ unsigned char used[QRC_LOC];
    __shared__ double coef[QRC_LOC];
    __shared__ double offer_v[2];
    __shared__ int offer_c[2];
    __shared__ double red[QRC_THREADS / 32];
    __shared__ int s_piv;
    __shared__ double s_best, s_inv;
    const int p = D.p, l = D.l, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    double *const mine = gscr ? gscr + (size_t)blockIdx.x * 3 * pstride : smx;
    double *qv = mine, *part = mine + p;
    // global mode: the first CTA of this cluster's vectors (rank q's are q * 3 pstride on)
    const double *gbase = gscr ? gscr + (size_t)(blockIdx.x - cr) * 3 * pstride + p : nullptr;
    const int nloc = cr < l ? (l - cr + cs - 1) / cs : 0;
    // my columns into the work copy, with their norms
    for (int i = warp; i < nloc; i += nw) {
        const int g = cr + cs * i;
        const double *a = D.A + (size_t)g * D.lda;
        double *w = D.W + (size_t)g * p;
        double s = 0.0;
        for (int x = lane; x < p; x += 32) {
            const double v = a[x];
            __stcg(w + x, v);
            s = fma(v, v, s);
        }
        s = warp_sum_d(s);
        if (lane == 0) {
            nrm[i] = s;
            used[i] = 0;
        }
    }
    __syncthreads();
    int ktr = -1, kval = 0;
    double r11 = 0.0;
    const int steps = min(kmax, min(p, l));
    for (int j = 0; j < steps; ++j) {
        const int buf = j & 1;
        if (warp == 0) {  // my offer: largest unused norm, lowest column on ties
            double bv = -1.0;
            int bc = 0x7fffffff;
            for (int i = lane; i < nloc; i += 32)
                if (!used[i] && nrm[i] > bv) {
                    bv = nrm[i];
                    bc = cr + cs * i;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
                if (ov > bv || (ov == bv && oc < bc)) {
                    bv = ov;
                    bc = oc;
                }
            }
            if (lane == 0) {
                offer_v[buf] = bv;
                offer_c[buf] = bc;
            }
        }
        cl.sync();
        if (tid == 0) {
            double bv = -1.0;
            int bc = 0x7fffffff;
            for (int q = 0; q < cs; ++q) {
                const double v = *cl.map_shared_rank(&offer_v[buf], q);
                const int c = *cl.map_shared_rank(&offer_c[buf], q);
                if (v > bv || (v == bv && c < bc)) {
                    bv = v;
                    bc = c;
                }
            }
            s_piv = bv >= 0.0 ? bc : -1;
            s_best = bv;
        }
        __syncthreads();
        const int pv = s_piv;
        const double rjj = s_best > 0.0 ? sqrt(s_best) : 0.0;
        if (j == 0) r11 = rjj;
        if (ktr < 0 && !(rjj > tol * r11)) ktr = j;
        if (pv < 0 || !(rjj > 1e-15 * r11) || !(r11 > 0.0) || (ktr >= 0 && j >= ktr + margin)) break;
        const double *wp = D.W + (size_t)pv * p;
        for (int x = tid; x < p; x += blockDim.x) qv[x] = __ldcg(wp + x);
        __syncthreads();
        // my part of Q (Q^T a): the columns t of Q with t = cr (mod cs), t < j
        const int nq = j > cr ? (j - cr + cs - 1) / cs : 0;
        for (int t = warp; t < nq; t += nw) {
            const double *qc = D.Q + (size_t)(cr + cs * t) * D.ldq;
            double s = 0.0;
            for (int x = lane; x < p; x += 32) s = fma(__ldcg(qc + x), qv[x], s);
            s = warp_sum_d(s);
            if (lane == 0) coef[t] = s;
        }
        __syncthreads();
        double *pb = part + (size_t)buf * p;
        for (int x = tid; x < p; x += blockDim.x) {
            double v = 0.0;
            for (int t = 0; t < nq; ++t) v = fma(coef[t], __ldcg(D.Q + x + (size_t)(cr + cs * t) * D.ldq), v);
            if (gscr) __stcg(pb + x, v);
            else pb[x] = v;
        }
        if (gscr) __threadfence();
        cl.sync();
        double ss = 0.0;
        for (int x = tid; x < p; x += blockDim.x) {
            double v = qv[x];
            if (gscr) {
                for (int q = 0; q < cs; ++q) v -= __ldcg(gbase + (size_t)q * 3 * pstride + (size_t)buf * p + x);
            } else {
                for (int q = 0; q < cs; ++q) v -= cl.map_shared_rank(pb, q)[x];
            }
            qv[x] = v;
            ss = fma(v, v, ss);
        }
        ss = warp_sum_d(ss);
        if (lane == 0) red[warp] = ss;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[w];
            s_inv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
        }
        __syncthreads();
        const double inv = s_inv;
        const bool owner = pv % cs == cr;
        for (int x = tid; x < p; x += blockDim.x) {
            const double v = qv[x] * inv;
            qv[x] = v;
            if (owner) __stcg(D.Q + x + (size_t)j * D.ldq, v);
        }
        if (owner && tid == 0) used[pv / cs] = 1;
        __syncthreads();
        // remove q from my unused columns, refresh their norms
        for (int i = warp; i < nloc; i += nw) {
            if (used[i]) continue;
            double *w = D.W + (size_t)(cr + cs * i) * p;
            double s = 0.0;
            for (int x = lane; x < p; x += 32) s = fma(qv[x], __ldcg(w + x), s);
            s = warp_sum_d(s);
            double nn = 0.0;
            for (int x = lane; x < p; x += 32) {
                const double v = fma(-s, qv[x], __ldcg(w + x));
                __stcg(w + x, v);
                nn = fma(v, v, nn);
            }
            nn = warp_sum_d(nn);
            if (lane == 0) nrm[i] = nn;
        }
        __syncthreads();
        kval = j + 1;
    }
    if (cr == 0 && tid == 0) {
        D.out[0] = ktr < 0 ? kval : ktr;
        D.out[1] = kval;
    }
    cl.sync();
}

// With c == nullptr, b is a table of five weights per node (a conductance network).
__device__ __forceinline__ double stencil_w_h(const double *__restrict__ b, const double *__restrict__ c,
                                              const double *__restrict__ d, double ih, int g, int dir) {
    if (!c) return b[5 * (int64_t)g + dir];
    const double ih2 = ih * ih;  // ih = 1/h = n+1 exactly
    switch (dir) {
    case DIR_E: return -ih2 + b[g] * ih;
    case DIR_W: return -ih2 - b[g] * ih;
    case DIR_N: return -ih2 + c[g] * ih;
    default: return -ih2 - c[g] * ih;
    }
}

// Ghost k: its ring neighbour's global node and the direction from that node to k.
__device__ __forceinline__ void ghost_of(int n, int k, int &g, int &dir) {
    const int side = k / n, t = k % n;
    if (side == 0) { g = t; dir = DIR_S; }
    else if (side == 1) { g = (n - 1) + n * t; dir = DIR_E; }
    else if (side == 2) { g = (n - 1 - t) + n * (n - 1); dir = DIR_N; }
    else { g = n * (n - 1 - t); dir = DIR_W; }
}

// Coupling table of the root ring: node q couples to ghost k1 (and k2 at corners) with
// stencil weights w1 (w2); cp = [k1, k2] as ints and [w1, w2] as doubles per node.
__global__ void k_hbs_couple(int n, const double *__restrict__ bf, const double *__restrict__ cf,
                             const double *__restrict__ df, int *__restrict__ kk, double *__restrict__ ww) {
    const int r = 4 * n - 4;
    const double ih = n + 1.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < r; q += gridDim.x * blockDim.x) {
        // ring position of ghost k is k - floor(k/n) (mod r): sides share corner nodes
        const int s = q / (n - 1), t = q - s * (n - 1);
        const int k1 = s * n + t;
        int k2 = -1;
        if (t == 0) k2 = (s == 0) ? 4 * n - 1 : s * n - 1;
        int g, dir;
        ghost_of(n, k1, g, dir);
        kk[2 * q] = k1;
        ww[2 * q] = stencil_w_h(bf, cf, df, ih, g, dir);
        kk[2 * q + 1] = k2;
        double w2 = 0.0;
        if (k2 >= 0) {
            ghost_of(n, k2, g, dir);
            w2 = stencil_w_h(bf, cf, df, ih, g, dir);
        }
        ww[2 * q + 1] = w2;
    }
}

// x(q, j) = -(w1 g(k1, j) + w2 g(k2, j)): the ghost couplings moved to the right side.
__global__ void k_hbs_gather(int n, int B, const int *__restrict__ kk, const double *__restrict__ ww,
                             const double *__restrict__ g, double *__restrict__ x) {
    const int r = 4 * n - 4, N = 4 * n;
    const int64_t tot = (int64_t)r * B;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % r), j = (int)(e / r);
        double v = ww[2 * q] * g[kk[2 * q] + (size_t)j * N];
        if (kk[2 * q + 1] >= 0) v += ww[2 * q + 1] * g[kk[2 * q + 1] + (size_t)j * N];
        x[e] = -v;
    }
}

// dudn(k, j) = (g(k, j) - y(ring(k), j)) / h
__global__ void k_hbs_out(int n, int B, const double *__restrict__ g, const double *__restrict__ y,
                          double *__restrict__ out) {
    const int r = 4 * n - 4, N = 4 * n;
    const double ih = n + 1.0;
    const int64_t tot = (int64_t)N * B;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % N), j = (int)(e / N);
        int q = k - k / n;
        if (q >= r) q -= r;
        out[e] = (g[e] - y[q + (size_t)j * r]) * ih;
    }
}

// ----------------------------------------------------------------------------- host side

#define HCK(x)                                          \
    do {                                                \
        cudaError_t _e = (x);                           \
        if (_e != cudaSuccess) return GM_ECUDA;         \
    } while (0)

// Device staging for descriptor arrays (grown on demand, freed at the end of a call).
struct DescBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaStream_t s = nullptr;
    ~DescBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    int ensure(size_t bytes, cudaStream_t st) {
        s = st;
        if (bytes <= cap) return GM_OK;
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        cap = std::max(bytes, (size_t)64 * 1024);
        if (cudaMallocAsync(&p, cap, st) != cudaSuccess) {
            cudaGetLastError();
            cap = 0;
            return GM_ENOMEM;
        }
        return GM_OK;
    }
};

// Algorithmic flops of the HBS steps issued by this thread since the last take.
thread_local double tl_flops = 0.0;

int run_gemms(const std::vector<GemmDesc> &v, DescBuf &db, cudaStream_t s) {
    if (v.empty()) return GM_OK;
    for (const GemmDesc &d : v) tl_flops += 2.0 * d.m * d.n * d.k;
    int rc = db.ensure(v.size() * sizeof(GemmDesc), s);
    if (rc) return rc;
    HCK(cudaMemcpyAsync(db.p, v.data(), v.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, s));
    int mm = 0, nn = 0;
    for (const GemmDesc &d : v) {
        mm = std::max(mm, d.m);
        nn = std::max(nn, d.n);
    }
    if (mm == 0 || nn == 0) return GM_OK;
    for (size_t b0 = 0; b0 < v.size(); b0 += 65535) {
        const int cnt = (int)std::min<size_t>(65535, v.size() - b0);
        k_hgemm<<<dim3((mm + 63) / 64, (nn + 63) / 64, cnt), 256, 0, s>>>((const GemmDesc *)db.p + b0);
    }
    HCK(cudaGetLastError());
    return GM_OK;
}

int run_copies(const std::vector<CopyDesc> &v, DescBuf &db, cudaStream_t s) {
    if (v.empty()) return GM_OK;
    int rc = db.ensure(v.size() * sizeof(CopyDesc), s);
    if (rc) return rc;
    HCK(cudaMemcpyAsync(db.p, v.data(), v.size() * sizeof(CopyDesc), cudaMemcpyHostToDevice, s));
    int64_t mx = 1;
    for (const CopyDesc &d : v) mx = std::max<int64_t>(mx, (int64_t)d.rows * d.cols);
    const int bx = (int)std::min<int64_t>((mx + 255) / 256, 1024);
    k_hbs_copy<<<dim3(bx, (unsigned)v.size()), 256, 0, s>>>((const CopyDesc *)db.p);
    HCK(cudaGetLastError());
    return GM_OK;
}

GemmDesc gd(const double *A, int lda, int ta, const double *B, int ldb, int tb, double *C, int ldc, int m, int n, int k,
            double alpha, double beta) {
    GemmDesc d;
    d.A = A;
    d.B = B;
    d.C = C;
    d.m = m;
    d.n = n;
    d.k = k;
    d.lda = std::max(lda, 1);
    d.ldb = std::max(ldb, 1);
    d.ldc = std::max(ldc, 1);
    d.ta = ta;
    d.tb = tb;
    d.alpha = alpha;
    d.beta = beta;
    return d;
}

CopyDesc cpd(const double *src, int lds, double *dst, int ldd, int rows, int cols, int mode) {
    CopyDesc d;
    d.src = src;
    d.dst = dst;
    d.rows = rows;
    d.cols = cols;
    d.lds = std::max(lds, 1);
    d.ldd = std::max(ldd, 1);
    d.mode = mode;
    d.pad = 0;
    return d;
}

struct Bump {
    int64_t top = 0;
    int64_t take(int64_t n) {
        const int64_t at = top;
        top += (n + 31) / 32 * 32;  // 256-byte aligned slots
        return at;
    }
};

// Batched inversion of square matrices in place: each sys (m x 2m, ld m) holds [M | I];
// after the sweep its right half is M^{-1}.
int invert_batch(const std::vector<std::pair<double *, int>> &mats, cudaStream_t s) {
    std::vector<SysDesc> h;
    int max_m = 0, roff = 0, coff = 0;
    double *base = nullptr;  // offsets from the lowest address among the matrices
    for (const auto &mt : mats)
        if (mt.second > 0 && (!base || mt.first < base)) base = mt.first;
    for (size_t i = 0; i < mats.size(); ++i) {
        const int m = mats[i].second;
        if (m == 0) continue;
        h.push_back(SysDesc{(int64_t)(mats[i].first - base), m, 2 * m, (int)i, roff, coff, 0});
        roff += m;
        coff += 2 * m;
        max_m = std::max(max_m, m);
    }
    if (h.empty()) return GM_OK;
    for (const SysDesc &q : h) tl_flops += 2.0 * (double)q.m * q.m * q.m;  // Gauss-Jordan on [M | I]
    const int nb = 8, nsys = (int)h.size();
    void *dsys = nullptr, *piv = nullptr, *u12 = nullptr, *st = nullptr;
    int rc = GM_OK;
    if (cudaMallocAsync(&dsys, h.size() * sizeof(SysDesc), s) != cudaSuccess ||
        cudaMallocAsync(&piv, (size_t)nsys * max_m * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync(&u12, (size_t)nsys * nb * 2 * max_m * sizeof(double), s) != cudaSuccess ||
        cudaMallocAsync(&st, sizeof(Status), s) != cudaSuccess) {
        cudaGetLastError();
        rc = GM_ENOMEM;
    }
    Status st0{0, -1, 0x7ff0000000000000ull, 0, 0u}, st1{};
    if (rc == GM_OK) {
        KTimer kt;
        if (cudaMemcpyAsync(dsys, h.data(), h.size() * sizeof(SysDesc), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(st, &st0, sizeof(st0), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            launch_gj_sweep((const SysDesc *)dsys, h, max_m, 2 * max_m, base, nb, (int *)piv, max_m, (double *)u12,
                            (int64_t)nb * 2 * max_m, (Status *)st, 0, s, kt) != cudaSuccess ||
            cudaMemcpyAsync(&st1, st, sizeof(st1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = GM_ECUDA;
        else if (st1.code)
            rc = st1.code;
    }
    for (void *p : {dsys, piv, u12, st})
        if (p) cudaFreeAsync(p, s);
    return rc;
}

// Temporary device buffers of one call, from the library pool, released on scope exit.
struct TempSet {
    cudaStream_t s;
    std::vector<void *> v;
    explicit TempSet(cudaStream_t st) : s(st) {}
    TempSet(const TempSet &) = delete;
    TempSet &operator=(const TempSet &) = delete;
    ~TempSet() {
        for (void *p : v) cudaFreeAsync(p, s);
    }
    double *get(int64_t doubles) {
        void *p = nullptr;
        if (dev_alloc(&p, (size_t)std::max<int64_t>(doubles, 1) * 8, s) != GM_OK) return nullptr;
        v.push_back(p);
        return (double *)p;
    }
};

// Largest dynamic shared memory of the single-CTA factorisation.
size_t qr_smem(int p, int l) { return (size_t)p * l * sizeof(double); }

// One level of pivoted QR factorisations (k_hbs_pqr or the cluster kernel, by size).
int run_qr(const std::vector<QrDesc> &q, double tol, int margin, DescBuf &db, cudaStream_t s) {
    if (q.empty()) return GM_OK;
    int maxp = 0, maxl = 0;
    for (const QrDesc &d : q) {
        maxp = std::max(maxp, d.p);
        maxl = std::max(maxl, d.l);
    }
    if (maxp > QRC_MAXP_G || maxl > HBS_MAX_SAMPLES) return GM_EUNSUPPORTED;
    int rc = db.ensure(q.size() * sizeof(QrDesc), s);
    if (rc) return rc;
    HCK(cudaMemcpyAsync(db.p, q.data(), q.size() * sizeof(QrDesc), cudaMemcpyHostToDevice, s));
    const int kmax = std::max(maxp, maxl);
    if (maxp <= QR_MAXP && maxl <= HBS_SAMPLES) {
        const size_t sm = qr_smem(maxp, maxl);
        HCK(raise_smem_limit((const void *)k_hbs_pqr, sm));  // the merges' threads share the limit
        k_hbs_pqr<<<(unsigned)q.size(), 256, sm, s>>>((const QrDesc *)db.p, tol, kmax, margin);
        HCK(cudaGetLastError());
        return GM_OK;
    }
    // samples taller than QRC_MAXP rows keep the per-CTA vectors in global memory (for at
    // most 16 CTAs per factorisation)
    const bool glob = maxp > QRC_MAXP;
    double *gscr = nullptr;
    if (glob && cudaMallocAsync((void **)&gscr, q.size() * 16 * 3 * (size_t)maxp * sizeof(double), s) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    const size_t sm = glob ? 0 : (size_t)3 * maxp * sizeof(double);
    HCK(raise_smem_limit((const void *)k_hbs_pqr_cl, sm));
    HCK(cudaFuncSetAttribute(k_hbs_pqr_cl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaError_t e = cudaErrorInvalidValue;
    for (int cs : {16, 8}) {  // 16 CTAs where the device schedules such clusters, else 8
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(q.size() * cs));
        cfg.blockDim = dim3(QRC_THREADS);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_hbs_pqr_cl, (const QrDesc *)db.p, tol, kmax, margin, gscr, maxp);
        if (e == cudaSuccess) break;
        cudaGetLastError();
    }
    if (gscr) cudaFreeAsync(gscr, s);
    return e == cudaSuccess ? GM_OK : GM_ECUDA;
}

// Sample counts for a size class (r rounded up to a power of two, node size m): the
// count the last factorisation of that class needed for its ranks, so that later builds
// of the same workload start there and a lower-rank workload after a higher-rank one
// drops back after its first factorisation.
std::mutex g_hint_mu;
std::map<std::pair<int, int>, int> g_hint;
// Inside hbs_hints_freeze / hbs_hints_thaw (merges factorised concurrently) a thread reads
// the hints of the snapshot taken at freeze and records its own in tl_hint_out, so that
// every merge starts from the same counts whatever the order the threads run in.
std::map<std::pair<int, int>, int> g_hint_frozen;
bool g_hint_is_frozen = false;
thread_local std::map<std::pair<int, int>, int> *tl_hint_out = nullptr;

int hint_get(const std::pair<int, int> &key, int dflt) {
    std::lock_guard<std::mutex> lk(g_hint_mu);
    const auto &m = g_hint_is_frozen ? g_hint_frozen : g_hint;
    auto it = m.find(key);
    return it != m.end() ? it->second : dflt;
}

void hint_set(const std::pair<int, int> &key, int v) {
    if (tl_hint_out) {
        (*tl_hint_out)[key] = v;
        return;
    }
    std::lock_guard<std::mutex> lk(g_hint_mu);
    g_hint[key] = v;
}

// The smallest count of the doubling sequence from HBS_SAMPLES that leaves HBS_OVERSAMPLE
// columns beyond `rank`.
int samples_for(int rank) {
    int l = HBS_SAMPLES;
    while (l < HBS_MAX_SAMPLES && rank > l - HBS_OVERSAMPLE) l *= 2;
    return std::min(l, HBS_MAX_SAMPLES);
}

int size_class(int r) {
    int c = 1;
    while (c < r) c <<= 1;
    return c;
}

constexpr int HBS_RETRY = 1000;  // internal: more samples are needed

// One attempt of the compression with l samples per node, then Algorithm 1.
int hbs_factor_l(const double *S, int lds, int r, int m, double tol, int l, bool temp, cudaStream_t s, HbsRoot &H) {
    H.r = r;
    H.m = m;
    H.tol = tol;
    int L = 0;
    while ((r + (1 << L) - 1) / (1 << L) > m) ++L;
    if (L < 1) return GM_EUNSUPPORTED;  // a single node: nothing to compress
    H.L = L;
    const int NN = 1 << (L + 1);
    H.lo.assign(NN, 0);
    H.hi.assign(NN, 0);
    H.k.assign(NN, 0);
    H.max_rank = 0;
    H.max_trunc = 0;
    H.lo[1] = 0;
    H.hi[1] = r;
    for (int t = 1; t < (1 << L); ++t) {
        const int mid = H.lo[t] + (H.hi[t] - H.lo[t]) / 2;
        H.lo[2 * t] = H.lo[t];
        H.hi[2 * t] = mid;
        H.lo[2 * t + 1] = mid;
        H.hi[2 * t + 1] = H.hi[t];
    }
    auto sz = [&](int t) { return H.hi[t] - H.lo[t]; };
    auto leaf = [&](int t) { return t >= (1 << L); };
    TempSet tmp(s);
    DescBuf db;
    int rc;
    double *Om = tmp.get((int64_t)r * l), *Ps = tmp.get((int64_t)r * l);
    double *Y = tmp.get((int64_t)r * l), *Z = tmp.get((int64_t)r * l);
    int *outs = (int *)tmp.get(2 * (int64_t)NN);  // per node: 2 QR results for U, 2 for V (ints)
    if (!Om || !Ps || !Y || !Z || !outs) return GM_ENOMEM;
    std::vector<double *> U(NN), V(NN), Uf(NN), Vf(NN), Ys(NN), Zs(NN), yr(NN), zr(NN);
    std::vector<double *> Hab(NN), Hba(NN), Wab(NN), Wba(NN), Xab(NN), Xba(NN);
    auto rows_of = [&](int t) { return leaf(t) ? sz(t) : H.k[2 * t] + H.k[2 * t + 1]; };

    // ---- samples Y = S Omega, Z = S^T Psi
    k_hbs_normals<<<256, 256, 0, s>>>(Om, (int64_t)r * l, 0x4842530000000001ull);
    k_hbs_normals<<<256, 256, 0, s>>>(Ps, (int64_t)r * l, 0x4842530000000002ull);
    HCK(cudaGetLastError());
    if ((rc = run_gemms({gd(S, lds, 0, Om, r, 0, Y, r, r, l, r, 1.0, 0.0), gd(S, lds, 1, Ps, r, 0, Z, r, r, l, r, 1.0, 0.0)},
                        db, s)))
        return rc;

    // QR of the samples of one level: rank of each node = the larger truncation point of
    // its two bases, within the columns both produced; a rank within HBS_OVERSAMPLE of the
    // sample count asks for more samples
    auto qr_level = [&](const std::vector<int> &nodes) -> int {
        std::vector<QrDesc> q;
        for (int t : nodes) {
            const int p = rows_of(t), kc = std::min(p, l);
            U[t] = tmp.get((int64_t)p * kc);
            V[t] = tmp.get((int64_t)p * kc);
            double *w1 = tmp.get((int64_t)p * l), *w2 = tmp.get((int64_t)p * l);
            if (!U[t] || !V[t] || !w1 || !w2) return GM_ENOMEM;
            q.push_back(QrDesc{Ys[t], U[t], outs + 4 * t, w1, p, l, p, p});
            q.push_back(QrDesc{Zs[t], V[t], outs + 4 * t + 2, w2, p, l, p, p});
        }
        int rc2 = run_qr(q, tol, HBS_MARGIN, db, s);
        if (rc2) return rc2;
        for (const QrDesc &d : q) tl_flops += 4.0 * d.p * d.l * std::min(d.p, d.l) / 2;  // half the steps, on average
        // the nodes of a level are consecutive: one read-back
        const int t0 = nodes.front(), cnt = nodes.back() - t0 + 1;
        std::vector<int> res(4 * (size_t)cnt);
        HCK(cudaMemcpyAsync(res.data(), outs + 4 * t0, res.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        HCK(cudaStreamSynchronize(s));
        for (int t : nodes) {
            const int *o = &res[4 * (size_t)(t - t0)];
            const int tu = o[0], pu = o[1], tv = o[2], pv = o[3];
            const int kt = std::min(std::max(tu, tv), std::min(pu, pv));
            // a rank close to the sample count: the samples may have missed part of the range
            if (std::max(tu, tv) > l - HBS_OVERSAMPLE && l < std::min(rows_of(t), sz(1) - sz(t))) return HBS_RETRY;
            H.k[t] = kt;
            H.max_rank = std::max(H.max_rank, kt);
            H.max_trunc = std::max(H.max_trunc, std::max(tu, tv));
        }
        return GM_OK;
    };

    // ---- leaves: sample of the off-diagonal block row / column, bases, reduced samples
    {
        std::vector<CopyDesc> cp;
        std::vector<GemmDesc> g;
        std::vector<int> nodes;
        for (int t = 1 << L; t < NN; ++t) {
            const int lo = H.lo[t], p = sz(t);
            Ys[t] = tmp.get((int64_t)p * l);
            Zs[t] = tmp.get((int64_t)p * l);
            if (!Ys[t] || !Zs[t]) return GM_ENOMEM;
            const double *Sd = S + lo + (size_t)lo * lds;
            cp.push_back(cpd(Y + lo, r, Ys[t], p, p, l, 0));
            cp.push_back(cpd(Z + lo, r, Zs[t], p, p, l, 0));
            g.push_back(gd(Sd, lds, 0, Om + lo, r, 0, Ys[t], p, p, l, p, -1.0, 1.0));
            g.push_back(gd(Sd, lds, 1, Ps + lo, r, 0, Zs[t], p, p, l, p, -1.0, 1.0));
            nodes.push_back(t);
        }
        if ((rc = run_copies(cp, db, s)) || (rc = run_gemms(g, db, s)) || (rc = qr_level(nodes))) return rc;
        g.clear();
        for (int t : nodes) {
            const int p = sz(t), k = H.k[t];
            yr[t] = tmp.get((int64_t)k * l);
            zr[t] = tmp.get((int64_t)k * l);
            if (!yr[t] || !zr[t]) return GM_ENOMEM;
            Uf[t] = U[t];
            Vf[t] = V[t];
            g.push_back(gd(U[t], p, 1, Ys[t], p, 0, yr[t], std::max(k, 1), k, l, p, 1.0, 0.0));
            g.push_back(gd(V[t], p, 1, Zs[t], p, 0, zr[t], std::max(k, 1), k, l, p, 1.0, 0.0));
        }
        if ((rc = run_gemms(g, db, s))) return rc;
    }
    // ---- parents, finest first; the root (level 0) only needs its B blocks
    for (int lev = L - 1; lev >= 0; --lev) {
        std::vector<GemmDesc> g1, g2;
        std::vector<CopyDesc> cp;
        std::vector<int> nodes;
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int a = 2 * t, b = 2 * t + 1, ka = H.k[a], kb = H.k[b];
            const int sa = sz(a), sb = sz(b);
            Wab[t] = tmp.get((int64_t)ka * sb);
            Wba[t] = tmp.get((int64_t)kb * sa);
            Xab[t] = tmp.get((int64_t)sa * kb);
            Xba[t] = tmp.get((int64_t)sb * ka);
            Hab[t] = tmp.get((int64_t)ka * kb);
            Hba[t] = tmp.get((int64_t)kb * ka);
            if (!Wab[t] || !Wba[t] || !Xab[t] || !Xba[t] || !Hab[t] || !Hba[t]) return GM_ENOMEM;
            const double *Sab = S + H.lo[a] + (size_t)H.lo[b] * lds, *Sba = S + H.lo[b] + (size_t)H.lo[a] * lds;
            // W_ab = Uf_a^T S(I_a, I_b), W_ba = Uf_b^T S(I_b, I_a)
            g1.push_back(gd(Uf[a], sa, 1, Sab, lds, 0, Wab[t], std::max(ka, 1), ka, sb, sa, 1.0, 0.0));
            g1.push_back(gd(Uf[b], sb, 1, Sba, lds, 0, Wba[t], std::max(kb, 1), kb, sa, sb, 1.0, 0.0));
            // X_ab = S(I_a, I_b) Vf_b, X_ba = S(I_b, I_a) Vf_a
            g1.push_back(gd(Sab, lds, 0, Vf[b], sb, 0, Xab[t], sa, sa, kb, sb, 1.0, 0.0));
            g1.push_back(gd(Sba, lds, 0, Vf[a], sa, 0, Xba[t], sb, sb, ka, sa, 1.0, 0.0));
            // B_tau blocks: H_ab = W_ab Vf_b, H_ba = W_ba Vf_a
            g2.push_back(gd(Wab[t], std::max(ka, 1), 0, Vf[b], sb, 0, Hab[t], std::max(ka, 1), ka, kb, sb, 1.0, 0.0));
            g2.push_back(gd(Wba[t], std::max(kb, 1), 0, Vf[a], sa, 0, Hba[t], std::max(kb, 1), kb, ka, sa, 1.0, 0.0));
            if (lev >= 1) {
                const int p = ka + kb;
                Ys[t] = tmp.get((int64_t)p * l);
                Zs[t] = tmp.get((int64_t)p * l);
                if (!Ys[t] || !Zs[t]) return GM_ENOMEM;
                // reduced samples: [y_a - W_ab Omega(I_b); y_b - W_ba Omega(I_a)], same for z
                cp.push_back(cpd(yr[a], std::max(ka, 1), Ys[t], std::max(p, 1), ka, l, 0));
                cp.push_back(cpd(yr[b], std::max(kb, 1), Ys[t] + ka, std::max(p, 1), kb, l, 0));
                cp.push_back(cpd(zr[a], std::max(ka, 1), Zs[t], std::max(p, 1), ka, l, 0));
                cp.push_back(cpd(zr[b], std::max(kb, 1), Zs[t] + ka, std::max(p, 1), kb, l, 0));
                g2.push_back(gd(Wab[t], std::max(ka, 1), 0, Om + H.lo[b], r, 0, Ys[t], std::max(p, 1), ka, l, sb, -1.0,
                                1.0));
                g2.push_back(gd(Wba[t], std::max(kb, 1), 0, Om + H.lo[a], r, 0, Ys[t] + ka, std::max(p, 1), kb, l, sa,
                                -1.0, 1.0));
                g2.push_back(gd(Xba[t], sb, 1, Ps + H.lo[b], r, 0, Zs[t], std::max(p, 1), ka, l, sb, -1.0, 1.0));
                g2.push_back(gd(Xab[t], sa, 1, Ps + H.lo[a], r, 0, Zs[t] + ka, std::max(p, 1), kb, l, sa, -1.0, 1.0));
                nodes.push_back(t);
            }
        }
        if ((rc = run_gemms(g1, db, s)) || (rc = run_copies(cp, db, s)) || (rc = run_gemms(g2, db, s))) return rc;
        if (lev == 0) break;
        if ((rc = qr_level(nodes))) return rc;
        std::vector<GemmDesc> g3;
        for (int t : nodes) {
            const int a = 2 * t, b = 2 * t + 1, ka = H.k[a], kb = H.k[b], k = H.k[t], p = ka + kb;
            const int sa = sz(a), st = sz(t);
            yr[t] = tmp.get((int64_t)k * l);
            zr[t] = tmp.get((int64_t)k * l);
            Uf[t] = tmp.get((int64_t)st * k);
            Vf[t] = tmp.get((int64_t)st * k);
            if (!yr[t] || !zr[t] || !Uf[t] || !Vf[t]) return GM_ENOMEM;
            g3.push_back(gd(U[t], std::max(p, 1), 1, Ys[t], std::max(p, 1), 0, yr[t], std::max(k, 1), k, l, p, 1.0, 0.0));
            g3.push_back(gd(V[t], std::max(p, 1), 1, Zs[t], std::max(p, 1), 0, zr[t], std::max(k, 1), k, l, p, 1.0, 0.0));
            // full bases: Uf_t = diag(Uf_a, Uf_b) U_t, likewise V
            g3.push_back(gd(Uf[a], sa, 0, U[t], std::max(p, 1), 0, Uf[t], st, sa, k, ka, 1.0, 0.0));
            g3.push_back(gd(Uf[b], sz(b), 0, U[t] + ka, std::max(p, 1), 0, Uf[t] + sa, st, sz(b), k, kb, 1.0, 0.0));
            g3.push_back(gd(Vf[a], sa, 0, V[t], std::max(p, 1), 0, Vf[t], st, sa, k, ka, 1.0, 0.0));
            g3.push_back(gd(Vf[b], sz(b), 0, V[t] + ka, std::max(p, 1), 0, Vf[t] + sa, st, sz(b), k, kb, 1.0, 0.0));
        }
        if ((rc = run_gemms(g3, db, s))) return rc;
    }

    // ---- the factors that stay: E, F^T, G per node, G_1, the ring's ghost couplings
    Bump bp;
    H.offE.assign(NN, 0);
    H.offFt.assign(NN, 0);
    H.offG.assign(NN, 0);
    for (int t = 2; t < NN; ++t) {
        const int q = rows_of(t), k = H.k[t];
        H.offE[t] = bp.take((int64_t)q * k);
        H.offFt[t] = bp.take((int64_t)k * q);
        H.offG[t] = bp.take((int64_t)q * q);
    }
    const int q1 = H.k[2] + H.k[3];
    H.offG1 = bp.take((int64_t)q1 * 2 * q1);
    H.offKK = bp.take(r);
    H.offWW = bp.take(2 * (int64_t)r);
    H.pool_doubles = bp.top;
    H.pool_stream = temp ? s : nullptr;
    if (temp) {
        if ((rc = dev_alloc((void **)&H.pool, (size_t)bp.top * 8, s))) return rc;
    } else if (cudaMalloc((void **)&H.pool, (size_t)bp.top * 8) != cudaSuccess) {
        cudaGetLastError();
        H.pool = nullptr;
        return GM_ENOMEM;
    }
    double *P = H.pool;

    // ---- Algorithm 1, finest level first
    std::vector<double *> Dq(NN), Wt(NN), Xt(NN), Zt(NN);
    for (int lev = L; lev >= 1; --lev) {
        std::vector<CopyDesc> cp;
        std::vector<std::pair<double *, int>> inv;
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            Dq[t] = tmp.get((int64_t)q * 2 * q);  // [D~ | I], q x 2q, ld q
            Wt[t] = tmp.get((int64_t)q * k);
            Xt[t] = tmp.get((int64_t)k * 2 * k);  // [V^T W | I]
            Zt[t] = tmp.get((int64_t)k * q);
            if (!Dq[t] || !Wt[t] || !Xt[t] || !Zt[t]) return GM_ENOMEM;
            if (leaf(t)) {
                cp.push_back(cpd(S + H.lo[t] + (size_t)H.lo[t] * lds, lds, Dq[t], q, q, q, 0));
            } else {
                const int a = 2 * t, b = 2 * t + 1, ka = H.k[a], kb = H.k[b];
                const double *Dha = Xt[a] + (size_t)ka * ka, *Dhb = Xt[b] + (size_t)kb * kb;
                cp.push_back(cpd(Dha, std::max(ka, 1), Dq[t], q, ka, ka, 0));
                cp.push_back(cpd(Hab[t], std::max(ka, 1), Dq[t] + (size_t)ka * q, q, ka, kb, 0));
                cp.push_back(cpd(Hba[t], std::max(kb, 1), Dq[t] + ka, q, kb, ka, 0));
                cp.push_back(cpd(Dhb, std::max(kb, 1), Dq[t] + ka + (size_t)ka * q, q, kb, kb, 0));
            }
            cp.push_back(cpd(nullptr, 1, Dq[t] + (size_t)q * q, q, q, q, 1));
            inv.push_back({Dq[t], q});
        }
        if ((rc = run_copies(cp, db, s)) || (rc = invert_batch(inv, s))) return rc;
        // W = D~^-1 U, X = V^T W (into [X | I]), then D^ = X^-1
        std::vector<GemmDesc> g;
        cp.clear();
        inv.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            const double *Di = Dq[t] + (size_t)q * q;
            g.push_back(gd(Di, q, 0, U[t], q, 0, Wt[t], q, q, k, q, 1.0, 0.0));
            cp.push_back(cpd(nullptr, 1, Xt[t] + (size_t)k * k, std::max(k, 1), k, k, 1));
            inv.push_back({Xt[t], k});
        }
        if ((rc = run_gemms(g, db, s))) return rc;
        g.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            g.push_back(gd(V[t], q, 1, Wt[t], q, 0, Xt[t], std::max(k, 1), k, k, q, 1.0, 0.0));
        }
        if ((rc = run_gemms(g, db, s)) || (rc = run_copies(cp, db, s)) || (rc = invert_batch(inv, s))) return rc;
        // E = W D^, Zt = V^T D~^-1, F^T = D^ Zt, G = D~^-1 - E Zt
        g.clear();
        cp.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            const double *Di = Dq[t] + (size_t)q * q, *Dh = Xt[t] + (size_t)k * k;
            g.push_back(gd(Wt[t], q, 0, Dh, std::max(k, 1), 0, P + H.offE[t], q, q, k, k, 1.0, 0.0));
            g.push_back(gd(V[t], q, 1, Di, q, 0, Zt[t], std::max(k, 1), k, q, q, 1.0, 0.0));
            cp.push_back(cpd(Di, q, P + H.offG[t], q, q, q, 0));
        }
        if ((rc = run_gemms(g, db, s)) || (rc = run_copies(cp, db, s))) return rc;
        g.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            const double *Dh = Xt[t] + (size_t)k * k;
            g.push_back(gd(Dh, std::max(k, 1), 0, Zt[t], std::max(k, 1), 0, P + H.offFt[t], std::max(k, 1), k, q, k,
                           1.0, 0.0));
            g.push_back(gd(P + H.offE[t], q, 0, Zt[t], std::max(k, 1), 0, P + H.offG[t], q, q, q, k, -1.0, 1.0));
        }
        if ((rc = run_gemms(g, db, s))) return rc;
    }
    // G_1 = [D^_2, B_23; B_32, D^_3]^{-1}
    {
        const int k2 = H.k[2], k3 = H.k[3], q = k2 + k3;
        double *D1 = P + H.offG1;
        std::vector<CopyDesc> cp{cpd(Xt[2] + (size_t)k2 * k2, std::max(k2, 1), D1, q, k2, k2, 0),
                                 cpd(Hab[1], std::max(k2, 1), D1 + (size_t)k2 * q, q, k2, k3, 0),
                                 cpd(Hba[1], std::max(k3, 1), D1 + k2, q, k3, k2, 0),
                                 cpd(Xt[3] + (size_t)k3 * k3, std::max(k3, 1), D1 + k2 + (size_t)k2 * q, q, k3, k3, 0),
                                 cpd(nullptr, 1, D1 + (size_t)q * q, q, q, q, 1)};
        if ((rc = run_copies(cp, db, s)) || (rc = invert_batch({{D1, q}}, s))) return rc;
    }
    HCK(cudaStreamSynchronize(s));
    return GM_OK;
}

}  // namespace

double hbs_flops_take() {
    const double f = tl_flops;
    tl_flops = 0.0;
    return f;
}

namespace {
void release_pool(HbsRoot &h) {
    if (h.pool) {
        if (h.pool_stream) cudaFreeAsync(h.pool, h.pool_stream);
        else cudaFree(h.pool);
    }
    h.pool = nullptr;
    h.pool_stream = nullptr;
}
}  // namespace

// A-posteriori check of an inverse from Algorithm 1: the algorithm inverts each node's
// diagonal block without pivoting across blocks, which is unstable when such a block is
// nearly singular even though S is not (strongly convective operators).  With x four
// Gaussian vectors and y = S^{-1} x by Algorithm 2, the relative residual
// max |S y - x| / max |x|; a stable inverse leaves a small multiple of tol.
int hbs_residual(const double *S, int lds, HbsRoot &H, cudaStream_t s, double *resid) {
    const int r = H.r, B = 4;
    TempSet tmp(s);
    DescBuf db;
    double *X = tmp.get((int64_t)r * B), *Y = tmp.get((int64_t)r * B);
    if (!X || !Y) return GM_ENOMEM;
    k_hbs_normals<<<64, 256, 0, s>>>(X, (int64_t)r * B, 0x4842530000000007ull);
    HCK(cudaGetLastError());
    std::vector<double> hx((size_t)r * B), hz((size_t)r * B);
    HCK(cudaMemcpyAsync(hx.data(), X, hx.size() * 8, cudaMemcpyDeviceToHost, s));
    int rc = hbs_solve(H, X, r, Y, r, B, s);
    if (rc == GM_OK) rc = run_gemms({gd(S, lds, 0, Y, r, 0, X, r, r, B, r, 1.0, -1.0)}, db, s);  // X := S Y - X
    if (rc) return rc;
    HCK(cudaMemcpyAsync(hz.data(), X, hz.size() * 8, cudaMemcpyDeviceToHost, s));
    HCK(cudaStreamSynchronize(s));
    double mx = 0.0, mr = 0.0;
    for (size_t i = 0; i < hx.size(); ++i) {
        mx = std::max(mx, std::fabs(hx[i]));
        mr = std::max(mr, std::isfinite(hz[i]) ? std::fabs(hz[i]) : 1e300);
    }
    *resid = mx > 0.0 ? mr / mx : 0.0;
    return GM_OK;
}

int hbs_factor(const double *S, int lds, int r, int m, double tol, cudaStream_t s, HbsRoot &H, bool temp) {
    if (r < 2 || lds < r || m < 2 || m > QR_MAXP || !(tol > 0.0)) return GM_EINVAL;
    const std::pair<int, int> key(size_class(r), m);
    int l = hint_get(key, HBS_SAMPLES);
    for (;;) {
        release_pool(H);
        const int rc = hbs_factor_l(S, lds, r, m, tol, l, temp, s, H);
        if (rc != HBS_RETRY) {
            if (rc == GM_OK) {
                hint_set(key, std::min(l, samples_for(H.max_trunc)));
                double res = 0.0;
                const int rc2 = hbs_residual(S, lds, H, s, &res);
                H.residual = res;
                if (rc2) return rc2;
                static const bool dbg = getenv("GM_DEBUG") != nullptr;
                if (dbg)
                    fprintf(stderr, "gm: hbs inverse r %d levels %d max rank %d tol %.1e: residual %.3e\n", r, H.L,
                            H.max_rank, tol, res);
                if (!(res <= HBS_MAX_RESIDUAL)) {  // unstable: the caller eliminates densely
                    release_pool(H);
                    return HBS_UNSTABLE;
                }
            }
            return rc;
        }
        if (l >= HBS_MAX_SAMPLES) {
            release_pool(H);
            return GM_EUNSUPPORTED;
        }
        l = std::min(2 * l, HBS_MAX_SAMPLES);
    }
}

int hbs_build_root(const double *S, int r, int n, int m, double tol, const double *bf, const double *cf,
                   const double *df, cudaStream_t s, HbsRoot &H) {
    int rc = hbs_factor(S, r, r, m, tol, s, H, false);
    if (rc) return rc;
    H.n = n;
    // coupling table for the solve
    k_hbs_couple<<<(r + 255) / 256, 256, 0, s>>>(n, bf, cf, df, (int *)(H.pool + H.offKK), H.pool + H.offWW);
    HCK(cudaGetLastError());
    HCK(cudaStreamSynchronize(s));
    return GM_OK;
}

int hbs_solve(HbsRoot &H, const double *X, int ldx, double *Y, int ldy, int B, cudaStream_t s) {
    if (B <= 0) return GM_OK;
    const int L = H.L, NN = 1 << (L + 1);
    auto leaf = [&](int t) { return t >= (1 << L); };
    // scratch: per parent the stacked x^ / y^ of its children
    Bump bp;
    std::vector<int64_t> oXs(NN, 0), oYs(NN, 0);
    std::vector<int> ks(NN, 0);
    for (int t = 1; t < (1 << L); ++t) {
        ks[t] = H.k[2 * t] + H.k[2 * t + 1];
        oXs[t] = bp.take((int64_t)std::max(ks[t], 1) * B);
        oYs[t] = bp.take((int64_t)std::max(ks[t], 1) * B);
    }
    double *W = nullptr;
    if (cudaMallocAsync((void **)&W, (size_t)bp.top * 8, s) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    const double *P = H.pool;
    DescBuf db;
    int rc = GM_OK;
    // where node t's x^ (and y^) live: rows [0, k_a) or [k_a, k_a + k_b) of its parent's stack
    auto xh = [&](int t) { return W + oXs[t / 2] + ((t & 1) ? H.k[t - 1] : 0); };
    auto yh = [&](int t) { return W + oYs[t / 2] + ((t & 1) ? H.k[t - 1] : 0); };
    auto ld = [&](int t) { return std::max(ks[t / 2], 1); };
    auto rows_of = [&](int t) { return leaf(t) ? H.hi[t] - H.lo[t] : ks[t]; };
    do {
        // up: x^_t = F_t^T x(I_t) at leaves, F_t^T [x^_a; x^_b] above
        std::vector<GemmDesc> v;
        for (int t = 1 << L; t < NN; ++t)
            v.push_back(gd(P + H.offFt[t], std::max(H.k[t], 1), 0, X + H.lo[t], ldx, 0, xh(t), ld(t), H.k[t], B,
                           rows_of(t), 1.0, 0.0));
        if ((rc = run_gemms(v, db, s))) break;
        for (int lev = L - 1; lev >= 1 && rc == GM_OK; --lev) {
            v.clear();
            for (int t = 1 << lev; t < (2 << lev); ++t)
                v.push_back(gd(P + H.offFt[t], std::max(H.k[t], 1), 0, W + oXs[t], std::max(ks[t], 1), 0, xh(t), ld(t),
                               H.k[t], B, ks[t], 1.0, 0.0));
            rc = run_gemms(v, db, s);
        }
        if (rc) break;
        // root: [y^_2; y^_3] = G_1 [x^_2; x^_3]
        if ((rc = run_gemms({gd(P + H.offG1 + (size_t)ks[1] * ks[1], std::max(ks[1], 1), 0, W + oXs[1],
                                std::max(ks[1], 1), 0, W + oYs[1], std::max(ks[1], 1), ks[1], B, ks[1], 1.0, 0.0)},
                             db, s)))
            break;
        // down: [y^_a; y^_b] = E_t y^_t + G_t [x^_a; x^_b]
        for (int lev = 1; lev < L && rc == GM_OK; ++lev) {
            std::vector<GemmDesc> v1, v2;
            for (int t = 1 << lev; t < (2 << lev); ++t) {
                const int q = ks[t];
                v1.push_back(gd(P + H.offE[t], std::max(q, 1), 0, yh(t), ld(t), 0, W + oYs[t], std::max(q, 1), q, B,
                                H.k[t], 1.0, 0.0));
                v2.push_back(gd(P + H.offG[t], std::max(q, 1), 0, W + oXs[t], std::max(q, 1), 0, W + oYs[t],
                                std::max(q, 1), q, B, q, 1.0, 1.0));
            }
            if ((rc = run_gemms(v1, db, s)) == GM_OK) rc = run_gemms(v2, db, s);
        }
        if (rc) break;
        // leaves: y(I_t) = E_t y^_t + G_t x(I_t)
        std::vector<GemmDesc> v1, v2;
        for (int t = 1 << L; t < NN; ++t) {
            const int q = rows_of(t);
            v1.push_back(gd(P + H.offE[t], q, 0, yh(t), ld(t), 0, Y + H.lo[t], ldy, q, B, H.k[t], 1.0, 0.0));
            v2.push_back(gd(P + H.offG[t], q, 0, X + H.lo[t], ldx, 0, Y + H.lo[t], ldy, q, B, q, 1.0, 1.0));
        }
        if ((rc = run_gemms(v1, db, s)) || (rc = run_gemms(v2, db, s))) break;
    } while (0);
    cudaFreeAsync(W, s);
    return rc;
}

int hbs_apply_dtn(HbsRoot &H, const double *g, double *dudn, int B, cudaStream_t s) {
    if (B <= 0) return GM_OK;
    const int r = H.r, n = H.n;
    double *W = nullptr;  // x = B g and y = S^{-1} x, r x B each
    if (cudaMallocAsync((void **)&W, (size_t)2 * r * B * 8, s) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    int rc = GM_OK;
    k_hbs_gather<<<256, 256, 0, s>>>(n, B, (const int *)(H.pool + H.offKK), H.pool + H.offWW, g, W);
    if (cudaGetLastError() != cudaSuccess) rc = GM_ECUDA;
    if (rc == GM_OK) rc = hbs_solve(H, W, r, W + (size_t)r * B, r, B, s);
    if (rc == GM_OK) {
        const int64_t tot = (int64_t)4 * n * B;
        k_hbs_out<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(n, B, g, W + (size_t)r * B, dudn);
        if (cudaGetLastError() != cudaSuccess) rc = GM_ECUDA;
    }
    if (rc == GM_OK && H.sig && launch_scale_rows(dudn, 4 * n, B, H.sig, s) != cudaSuccess) rc = GM_ECUDA;
    cudaFreeAsync(W, s);
    return rc;
}

namespace {
// D = Dsrc - diag(a) V (rows x cols; a read with stride sa)
__global__ void k_hbs_sub_diag(double *__restrict__ D, int ldd, const double *__restrict__ Dsrc, int ldsrc,
                               const double *__restrict__ a, int sa, const double *__restrict__ V, int ldv, int rows,
                               int cols) {
    const int64_t tot = (int64_t)rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % rows), j = (int)(e / rows);
        D[i + (size_t)j * ldd] = Dsrc[i + (size_t)j * ldsrc] - a[(size_t)i * sa] * V[i + (size_t)j * ldv];
    }
}
}  // namespace

int hbs_block_solve(double *ws, int sp, int rp, int m, double tol, cudaStream_t s, int *max_rank) {
    const int M = 2 * sp;
    HbsRoot H33, H44;
    double *T = nullptr;
    const size_t n1 = (size_t)sp * (sp + rp), n2 = (size_t)sp * sp, n3 = (size_t)sp * rp;
    if (cudaMallocAsync((void **)&T, (n1 + n2 + 3 * n3) * 8, s) != cudaSuccess) {
        cudaGetLastError();
        return GM_ENOMEM;
    }
    double *VW = T, *T44 = VW + n1, *Z4 = T44 + n2, *X4 = Z4 + n3, *X3 = X4 + n3;
    const double *V3 = VW, *W3 = VW + n2;
    int rc = GM_OK;
    DescBuf db;
    do {
        // S33 (top-left sp x sp of [M | Z]) in HBS form, inverted by Algorithm 1
        if ((rc = hbs_factor(ws, M, sp, m, tol, s, H33, true))) break;
        // [V3 W3] = S33^{-1} [A34 Z3]: the columns sp .. of the top rows of [M | Z]
        if ((rc = hbs_solve(H33, ws + (size_t)sp * M, M, VW, sp, sp + rp, s))) break;
        // T44 = S44 - A43 V3, Z4' = Z4 - A43 W3 (A43 diagonal: M(sp + i, i))
        const int bx = (int)std::min<int64_t>(((int64_t)sp * std::max(sp, rp) + 255) / 256, 4096);
        k_hbs_sub_diag<<<bx, 256, 0, s>>>(T44, sp, ws + sp + (size_t)sp * M, M, ws + sp, M + 1, V3, sp, sp, sp);
        k_hbs_sub_diag<<<bx, 256, 0, s>>>(Z4, sp, ws + sp + (size_t)M * M, M, ws + sp, M + 1, W3, sp, sp, rp);
        if (cudaGetLastError() != cudaSuccess) { rc = GM_ECUDA; break; }
        if ((rc = hbs_factor(T44, sp, sp, m, tol, s, H44, true))) break;
        if ((rc = hbs_solve(H44, Z4, sp, X4, sp, rp, s))) break;
        // X3 = W3 - V3 X4
        if ((rc = run_copies({cpd(W3, sp, X3, sp, sp, rp, 0)}, db, s))) break;
        if ((rc = run_gemms({gd(V3, sp, 0, X4, sp, 0, X3, sp, sp, rp, sp, -1.0, 1.0)}, db, s))) break;
        // X into the right block of [M | Z], as after the dense elimination
        if ((rc = run_copies({cpd(X3, sp, ws + (size_t)M * M, M, sp, rp, 0),
                              cpd(X4, sp, ws + sp + (size_t)M * M, M, sp, rp, 0)},
                             db, s)))
            break;
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = GM_ECUDA;
        if (max_rank) *max_rank = std::max(*max_rank, std::max(H33.max_rank, H44.max_rank));
    } while (0);
    hbs_free(H33);
    hbs_free(H44);
    cudaFreeAsync(T, s);
    return rc;
}

namespace {
// S13 = S1(P1, P3) and S24 = S2(P2, P4) of one merge, gathered from the children.
__global__ void k_hbs_gather_offdiag(const MergeDesc *__restrict__ md, const int *__restrict__ tab,
                                     const double *__restrict__ in, double *__restrict__ S13, double *__restrict__ S24) {
    const MergeDesc M = *md;
    const int sp = M.sp, n1 = M.n1, n2 = M.n2;
    const int *p3 = tab + M.tab, *p4 = p3 + sp, *p1 = p3 + 4 * sp, *p2 = p1 + 2 * n1;
    const double *S1 = in + M.s1, *S2 = in + M.s2;
    const int64_t t1 = (int64_t)n1 * sp, tot = t1 + (int64_t)n2 * sp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        if (e < t1) {
            const int a = (int)(e % n1), c = (int)(e / n1);
            S13[e] = S1[p1[a] + (int64_t)M.r1 * p3[c]];
        } else {
            const int64_t f = e - t1;
            const int a = (int)(f % n2), c = (int)(f / n2);
            S24[f] = S2[p2[a] + (int64_t)M.r2 * p4[c]];
        }
    }
}

// A_i ~ L_i R_i (A_i rows_i x cols, column-major, ld rows_i) at relative tolerance tol:
// L_i an orthonormal basis of the range of a Gaussian sample A_i Omega truncated at the
// first |R_jj| <= tol |R_11| of its pivoted QR, R_i = L_i^T A_i (k_i x cols).  The sample
// count starts at the one the last call for this size needed and doubles while a rank
// comes within HBS_OVERSAMPLE of it.  L_i, R_i come from tmp.
int lowrank_n(const std::vector<const double *> &A, const std::vector<int> &rows, int cols, double tol, TempSet &tmp,
              DescBuf &db, cudaStream_t s, std::vector<double *> &L, std::vector<double *> &R, std::vector<int> &k) {
    const size_t na = A.size();
    L.assign(na, nullptr);
    R.assign(na, nullptr);
    k.assign(na, 0);
    const std::pair<int, int> key(size_class(cols), -1);
    int l = hint_get(key, HBS_SAMPLES);
    int *outs = (int *)tmp.get((int64_t)na);
    if (!outs) return GM_ENOMEM;
    for (;;) {
        const int le = std::min(l, cols);
        double *Om = tmp.get((int64_t)cols * le);
        if (!Om) return GM_ENOMEM;
        k_hbs_normals<<<256, 256, 0, s>>>(Om, (int64_t)cols * le, 0x4842530000000003ull + (unsigned long long)l);
        HCK(cudaGetLastError());
        std::vector<GemmDesc> g;
        std::vector<QrDesc> q;
        for (size_t i = 0; i < na; ++i) {
            double *Y = tmp.get((int64_t)rows[i] * le);
            L[i] = tmp.get((int64_t)rows[i] * std::min(rows[i], le));
            double *w = tmp.get((int64_t)rows[i] * le);
            if (!Y || !L[i] || !w) return GM_ENOMEM;
            g.push_back(gd(A[i], rows[i], 0, Om, cols, 0, Y, rows[i], rows[i], le, cols, 1.0, 0.0));
            q.push_back(QrDesc{Y, L[i], outs + 2 * i, w, rows[i], le, rows[i], rows[i]});
        }
        int rc = run_gemms(g, db, s);
        if (rc == GM_OK) rc = run_qr(q, tol, 0, db, s);
        for (const QrDesc &d : q) tl_flops += 4.0 * d.p * d.l * std::min(d.p, d.l) / 2;
        if (rc) return rc;
        std::vector<int> res(2 * na);
        HCK(cudaMemcpyAsync(res.data(), outs, res.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        HCK(cudaStreamSynchronize(s));
        bool more = false;
        for (size_t i = 0; i < na; ++i) {
            k[i] = std::min(res[2 * i], res[2 * i + 1]);
            if (res[2 * i] > le - HBS_OVERSAMPLE && le < std::min(rows[i], cols)) more = true;
        }
        if (!more) break;
        if (l >= HBS_MAX_SAMPLES) return GM_EUNSUPPORTED;
        l = std::min(2 * l, HBS_MAX_SAMPLES);
    }
    {
        int kmax = 0;
        for (size_t i = 0; i < na; ++i) kmax = std::max(kmax, k[i]);
        hint_set(key, std::min(l, samples_for(kmax)));
    }
    std::vector<GemmDesc> g;
    for (size_t i = 0; i < na; ++i) {
        R[i] = tmp.get((int64_t)std::max(k[i], 1) * cols);
        if (!R[i]) return GM_ENOMEM;
        g.push_back(gd(L[i], rows[i], 1, A[i], rows[i], 0, R[i], std::max(k[i], 1), k[i], cols, rows[i], 1.0, 0.0));
    }
    return run_gemms(g, db, s);
}
}  // namespace

void hbs_hints_freeze() {
    std::lock_guard<std::mutex> lk(g_hint_mu);
    g_hint_frozen = g_hint;
    g_hint_is_frozen = true;
}

void hbs_hints_record(std::map<std::pair<int, int>, int> *out) { tl_hint_out = out; }

void hbs_hints_thaw(const std::vector<std::map<std::pair<int, int>, int>> &outs) {
    std::lock_guard<std::mutex> lk(g_hint_mu);
    for (const auto &m : outs)
        for (const auto &kv : m) g_hint[kv.first] = kv.second;  // in the callers' order
    g_hint_is_frozen = false;
}

int hbs_merge_lowrank(const MergeDesc &hm, const MergeDesc *d_md, const int *d_tab, const double *in,
                      const double *ws, double *out, const double *bf, const double *cf, const double *df, double tol,
                      cudaStream_t s, KTimer &kt, int *max_rank) {
    const int sp = hm.sp, rp = hm.rp, M = 2 * sp;
    TempSet tmp(s);
    DescBuf db;
    const int rows[2] = {hm.n1, hm.n2};
    double *S13 = tmp.get((int64_t)hm.n1 * sp), *S24 = tmp.get((int64_t)hm.n2 * sp);
    if (!S13 || !S24) return GM_ENOMEM;
    const int64_t tot = (int64_t)rp * sp;
    k_hbs_gather_offdiag<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(d_md, d_tab, in, S13, S24);
    HCK(cudaGetLastError());
    std::vector<double *> L, R;
    std::vector<int> k;
    int rc = lowrank_n({S13, S24}, {rows[0], rows[1]}, sp, tol, tmp, db, s, L, R, k);
    if (rc) return rc;
    // W13 = R13 X3, W24 = R24 X4 (X = M^{-1} Z, the right block of the system)
    const double *X = ws + (size_t)M * M;
    double *W13 = tmp.get((int64_t)std::max(k[0], 1) * rp), *W24 = tmp.get((int64_t)std::max(k[1], 1) * rp);
    if (!W13 || !W24) return GM_ENOMEM;
    if ((rc = run_gemms({gd(R[0], std::max(k[0], 1), 0, X, M, 0, W13, std::max(k[0], 1), k[0], rp, sp, 1.0, 0.0),
                         gd(R[1], std::max(k[1], 1), 0, X + sp, M, 0, W24, std::max(k[1], 1), k[1], rp, sp, 1.0, 0.0)},
                        db, s)))
        return rc;
    const LrUpdate lr{L[0], L[1], W13, W24, k[0], k[1]};
    HCK(launch_merge_update_lr(d_md, hm, d_tab, in, lr, out, bf, cf, df, s, kt));
    if (max_rank) *max_rank = std::max(*max_rank, std::max(k[0], k[1]));
    return GM_OK;
}

int hbs_lowrank(const double *A, int rows, int cols, double tol, cudaStream_t s, double **Lout, double **Rout,
                int *kout) {
    *Lout = *Rout = nullptr;
    *kout = 0;
    if (!A || rows < 1 || cols < 1 || !(tol > 0.0)) return GM_EINVAL;
    TempSet tmp(s);
    DescBuf db;
    std::vector<double *> L, R;
    std::vector<int> k;
    int rc = lowrank_n({A}, {rows}, cols, tol, tmp, db, s, L, R, k);
    if (rc) return rc;
    const int kk = k[0];
    if (cudaMalloc((void **)Lout, (size_t)rows * std::max(kk, 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)Rout, (size_t)std::max(kk, 1) * cols * 8) != cudaSuccess) {
        cudaGetLastError();
        if (*Lout) cudaFree(*Lout);
        *Lout = *Rout = nullptr;
        return GM_ENOMEM;
    }
    HCK(cudaMemcpyAsync(*Lout, L[0], (size_t)rows * kk * 8, cudaMemcpyDeviceToDevice, s));
    HCK(cudaMemcpyAsync(*Rout, R[0], (size_t)kk * cols * 8, cudaMemcpyDeviceToDevice, s));
    HCK(cudaStreamSynchronize(s));
    *kout = kk;
    return GM_OK;
}

int hbs_gemm(const double *A, int lda, int ta, const double *B, int ldb, int tb, double *C, int ldc, int m, int n,
             int k, double alpha, double beta, cudaStream_t s) {
    DescBuf db;
    return run_gemms({gd(A, lda, ta, B, ldb, tb, C, ldc, m, n, k, alpha, beta)}, db, s);
}

namespace {
__global__ void k_hbs_df2d(const float2 *__restrict__ x, double *__restrict__ y, int64_t cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (double)x[e].x + (double)x[e].y;
}
}  // namespace

cudaError_t hbs_df32_to_f64(const float2 *x, double *y, int64_t cnt, cudaStream_t s) {
    k_hbs_df2d<<<(int)std::min<int64_t>((cnt + 255) / 256, 4096), 256, 0, s>>>(x, y, cnt);
    return cudaGetLastError();
}

int hbs_dense_dtn(HbsRoot &H, double *T, cudaStream_t s) {
    // T = the solve applied to the identity, 512 columns at a time
    const int N = 4 * H.n, c = std::min(N, 512);
    double *G = nullptr, *V = nullptr;
    if (cudaMallocAsync((void **)&G, (size_t)N * c * 8, s) != cudaSuccess ||
        cudaMallocAsync((void **)&V, (size_t)N * c * 8, s) != cudaSuccess) {
        cudaGetLastError();
        if (G) cudaFreeAsync(G, s);
        return GM_ENOMEM;
    }
    int rc = GM_OK;
    DescBuf db;
    for (int j0 = 0; j0 < N && rc == GM_OK; j0 += c) {
        const int w = std::min(c, N - j0);
        // G(i, j) = [i == j0 + j]: identity columns j0 .. j0 + w - 1
        std::vector<CopyDesc> cp{cpd(nullptr, 1, G, N, N, w, 2), cpd(nullptr, 1, G + j0, N, w, w, 1)};
        if ((rc = run_copies({cp[0]}, db, s)) || (rc = run_copies({cp[1]}, db, s))) break;
        if ((rc = hbs_apply_dtn(H, G, V, w, s))) break;
        if (cudaMemcpyAsync(T + (size_t)j0 * N, V, (size_t)N * w * 8, cudaMemcpyDefault, s) != cudaSuccess)
            rc = GM_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GM_OK) rc = GM_ECUDA;
    cudaFreeAsync(G, s);
    cudaFreeAsync(V, s);
    return rc;
}

void hbs_free(HbsRoot &h) {
    if (h.pool) {
        if (h.pool_stream) cudaFreeAsync(h.pool, h.pool_stream);
        else cudaFree(h.pool);
    }
    h.pool = nullptr;
    h.pool_stream = nullptr;
    if (h.sig) cudaFree(h.sig);
    h.sig = nullptr;
}

}  // namespace gm
