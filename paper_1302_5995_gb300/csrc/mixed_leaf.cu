// Leaf Schur complement of the mixed-precision build (eq. def_schur_nd, Section 3.1):
//   S = A_bb - A_bi A_ii^{-1} A_ib
// with A_ii eliminated by banded Gaussian elimination with partial pivoting (Section 3.4
// cost remark), in double-float (df32) arithmetic on the FP32 units, the result written
// as df32 straight into the arena.  The FP64 build keeps k_leaf; this twin exists because
// GB300 issues a warp's FP64 instruction over many cycles, and the leaf's elimination is a
// chain of short dependent steps: in df32 every step is a few FP32 instructions instead.
//
// The interior unknowns are ordered i + ia j; A_bi and A_ib couple each non-corner ring
// node to exactly one interior node (an inner-ring node), so A_ii^{-1} is only needed at
// the inner-ring nodes: one unit right-hand side per inner-ring node.
#include <cuda_runtime.h>

#include <cstdint>

#include "gm_internal.h"
#include "kernels.h"
#include "mixed.h"
#include "mixed_dev.cuh"

namespace gm {

namespace {

// Ring position p (counter-clockwise from the box's SW corner) -> box coordinates.
__device__ __forceinline__ void ring_node_mx(int a, int b, int p, int &i, int &j) {
    if (p <= a - 1) { i = p; j = 0; }
    else if (p <= a + b - 2) { i = a - 1; j = p - a + 1; }
    else if (p <= 2 * a + b - 3) { i = 2 * a + b - 3 - p; j = b - 1; }
    else { i = 0; j = 2 * a + 2 * b - 4 - p; }
}

// Interior neighbour (interior coordinates) of the non-corner ring node (i, j) and the
// direction from the ring node to it; false for a corner.
__device__ __forceinline__ bool inner_nb(int a, int b, int i, int j, int &ii, int &jj, int &dir) {
    const int ib = b - 2;
    if (j == 0 && i > 0 && i < a - 1) { ii = i - 1; jj = 0; dir = DIR_N; return true; }
    if (j == b - 1 && i > 0 && i < a - 1) { ii = i - 1; jj = ib - 1; dir = DIR_S; return true; }
    if (i == 0 && j > 0 && j < b - 1) { ii = 0; jj = j - 1; dir = DIR_E; return true; }
    if (i == a - 1 && j > 0 && j < b - 1) { ii = a - 3; jj = j - 1; dir = DIR_W; return true; }
    return false;
}

__device__ __forceinline__ int opposite(int dir) {
    return dir == DIR_N ? DIR_S : dir == DIR_S ? DIR_N : dir == DIR_E ? DIR_W : DIR_E;
}

// df32 reciprocal: FP32 reciprocal and one Newton step on the df32 residual 1 - b r.
__device__ __forceinline__ float2 df_rcp(float2 b) {
    const float r = __frcp_rn(b.x);
    float e = fmaf(-b.x, r, 1.f);  // exact: 1 - b.x r is tiny
    e = fmaf(-b.y, r, e);
    return fast_two_sum(r, r * e);
}

// Magnitude bits of a pivot candidate (|hi| as an ordered integer; a NaN counts as 0).
__device__ __forceinline__ unsigned mag_bits(float2 v) {
    const float a = fabsf(v.x);
    return a == a ? __float_as_uint(a) : 0u;
}

}  // namespace

size_t mx_leaf_smem_bytes(int a, int b) {
    const int ia = a - 2, ib = b - 2;
    const int ni = (ia > 0 && ib > 0) ? ia * ib : 0;
    const int nq = ni == 0 ? 0 : (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
    const int W = 3 * (ia > 0 ? ia : 0) + 1, r = 2 * a + 2 * b - 4;
    return (size_t)ni * W * 8 + (size_t)ni * nq * 8 + (size_t)ni * 8 + (size_t)r * 6 * 8 +
           (size_t)(2 * ni + nq) * 4 + 16;
}

// One CTA per leaf (LEAF_THREADS threads).  Shared memory: the band of A_ii (ni x W,
// row q holds columns q - KL .. q + UW), the solves X (ni x nq), reciprocals of U's
// diagonal, six weights per ring node (C, E, W, N, S of its own equation, and the weight
// of its interior neighbour's equation on it), and the index maps.
__global__ void __launch_bounds__(LEAF_THREADS)
k_mx_leaf(const LeafDesc *__restrict__ leaves, const double *__restrict__ bf0, const double *__restrict__ cf0,
          const double *__restrict__ df0, float2 *__restrict__ out, Status *st, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LeafDesc Ld = leaves[blockIdx.x];
    const int n = Ld.n;
    const double *bf = bf0 + Ld.coef, *cf = cf0 + Ld.coef, *df = df0 + Ld.coef;
    const int a = Ld.a, bb = Ld.b;
    const int ia = a - 2, ib = bb - 2;
    const int ni = (ia > 0 && ib > 0) ? ia * ib : 0;
    const int r = 2 * a + 2 * bb - 4;
    const int KL = ia, UW = 2 * ia, W = 3 * ia + 1;
    const double ih = n + 1.0;  // 1/h
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    const int nq = ni == 0 ? 0 : (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
    float2 *band = (float2 *)smem_raw;  // ni * W
    float2 *X = band + (size_t)ni * W;  // ni * nq
    float2 *idg = X + (size_t)ni * nq;  // ni
    float2 *wr = idg + ni;              // r * 6
    int *piv = (int *)(wr + (size_t)r * 6);
    int *inner_id = piv + ni;  // ni
    int *inner_q = inner_id + ni;  // nq
    auto gnode = [&](int ii, int jj) { return (Ld.x0 + 1 + ii) + n * (Ld.y0 + 1 + jj); };
    auto band_at = [&](int row, int col) -> float2 & { return band[(size_t)row * W + KL + col - row]; };

    // weights of the ring nodes' equations (FP64 stencil, then df32)
    for (int l = tid; l < r; l += nt) {
        int il, jl;
        ring_node_mx(a, bb, l, il, jl);
        const int gl = (Ld.x0 + il) + n * (Ld.y0 + jl);
#pragma unroll
        for (int dir = 0; dir < 5; ++dir) wr[l * 6 + dir] = df_from_d(stencil_w_mx(bf, cf, df, ih, gl, dir));
        int ii, jj, dir;
        wr[l * 6 + 5] = (ni > 0 && inner_nb(a, bb, il, jl, ii, jj, dir))
                            ? df_from_d(stencil_w_mx(bf, cf, df, ih, gnode(ii, jj), opposite(dir)))
                            : make_float2(0.f, 0.f);
    }
    if (ni > 0) {
        for (int e = tid; e < ni * W; e += nt) band[e] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int q = tid; q < ni; q += nt) {
            const int ii = q % ia, jj = q / ia, g = gnode(ii, jj);
            band_at(q, q) = df_from_d(stencil_w_mx(bf, cf, df, ih, g, DIR_C));
            if (ii + 1 < ia) band_at(q, q + 1) = df_from_d(stencil_w_mx(bf, cf, df, ih, g, DIR_E));
            if (ii > 0) band_at(q, q - 1) = df_from_d(stencil_w_mx(bf, cf, df, ih, g, DIR_W));
            if (jj + 1 < ib) band_at(q, q + ia) = df_from_d(stencil_w_mx(bf, cf, df, ih, g, DIR_N));
            if (jj > 0) band_at(q, q - ia) = df_from_d(stencil_w_mx(bf, cf, df, ih, g, DIR_S));
            inner_id[q] = (ii == 0 || ii == ia - 1 || jj == 0 || jj == ib - 1) ? 1 : -1;
        }
        __syncthreads();
        if (tid == 0) {
            int c = 0;
            for (int q = 0; q < ni; ++q)
                if (inner_id[q] >= 0) { inner_id[q] = c; inner_q[c] = q; ++c; }
        }
        // Banded LU with partial pivoting (interchanges within the band).  Per column:
        // every warp finds the pivot row itself from the updated column (barrier: all
        // reads done), then the interchange and the multipliers (barrier), then the update
        // of the trailing band (barrier).
        // Until the first interchange row q reaches at most column q + KL, so the
        // elimination (and the backward sweep) can stop there.
        bool swapped = false;
        float2 pmin = make_float2(3.0e38f, 0.f);
        __syncthreads();
        for (int k = 0; k < ni; ++k) {
            const int last = min(k + KL, ni - 1);
            // pivot: the candidate (rows k .. last of column k) of largest |hi|, the lowest
            // row among equals; two warp reductions, done alike by every warp
            unsigned mb = 0u;
            for (int rr = k + lane; rr <= last; rr += 32) mb = max(mb, mag_bits(band_at(rr, k)));
            mb = __reduce_max_sync(0xffffffffu, mb);
            unsigned pr = 0xffffffffu;
            for (int rr = k + lane; rr <= last; rr += 32)
                if (mag_bits(band_at(rr, k)) == mb) pr = min(pr, (unsigned)rr);
            const int p = (int)__reduce_min_sync(0xffffffffu, pr);
            const float2 pv = band_at(p, k);
            swapped = swapped || p != k;
            const int cend = min(k + (swapped ? UW : KL), ni - 1);
            if (tid == 0) {
                piv[k] = p;
                if (fabsf(pv.x) < fabsf(pmin.x) || !(pv.x == pv.x)) pmin = pv;
            }
            // read everything this column step needs before anyone writes
            __syncthreads();
            if (p != k)
                for (int cc = k + 1 + tid; cc <= cend; cc += nt) {
                    const float2 x = band_at(k, cc);
                    band_at(k, cc) = band_at(p, cc);
                    band_at(p, cc) = x;
                }
            if (tid >= 1 && tid <= last - k) {  // column k: multipliers below the pivot
                const int rr = k + tid;
                const float2 ipv = df_rcp(pv);
                if (rr == p) {
                    const float2 old = band_at(k, k);
                    band_at(k, k) = pv;
                    band_at(p, k) = df_mul(old, ipv);
                } else {
                    band_at(rr, k) = df_mul(band_at(rr, k), ipv);
                }
            }
            __syncthreads();
            const int nr = last - k, ncn = cend - k;
            for (int e = tid; e < nr * ncn; e += nt) {
                const int rr = k + 1 + e / ncn, cc = k + 1 + e % ncn;
                band_at(rr, cc) = df_sub(band_at(rr, cc), df_mul(band_at(rr, k), band_at(k, cc)));
            }
            __syncthreads();
        }
        if (tid == 0) record_pivot_mx(st + Ld.prob, df_to_d(pmin), stage);
        const int UWe = swapped ? UW : KL;  // upper bandwidth of U
        for (int k = tid; k < ni; k += nt) idg[k] = df_rcp(band_at(k, k));
        for (int e = tid; e < ni * nq; e += nt) X[e] = make_float2(0.f, 0.f);
        __syncthreads();
        for (int t = tid; t < nq; t += nt) X[(size_t)inner_q[t] * nq + t] = make_float2(1.f, 0.f);
        __syncthreads();
        // forward and backward sweeps: the right-hand sides are independent, so each warp
        // owns up to 8 of them (lanes: 8 columns x 4 row slices) and syncs only itself
        {
            const int cpw = (nq + nwarp - 1) / nwarp;
            const int cl = lane & 7, rs = lane >> 3;
            for (int c0 = 0; c0 < cpw; c0 += 8) {
                const int t = warp * cpw + c0 + cl;
                const bool on = c0 + cl < cpw && t < nq;
                for (int k = 0; k < ni; ++k) {
                    const int p = piv[k];
                    if (on && rs == 0 && p != k) {
                        const float2 x0 = X[(size_t)k * nq + t];
                        X[(size_t)k * nq + t] = X[(size_t)p * nq + t];
                        X[(size_t)p * nq + t] = x0;
                    }
                    __syncwarp();
                    if (on) {
                        const int last = min(k + KL, ni - 1);
                        const float2 xk = X[(size_t)k * nq + t];
                        for (int rr = k + 1 + rs; rr <= last; rr += 4)
                            X[(size_t)rr * nq + t] = df_sub(X[(size_t)rr * nq + t], df_mul(band_at(rr, k), xk));
                    }
                    __syncwarp();
                }
                for (int k = ni - 1; k >= 0; --k) {
                    if (on && rs == 0) X[(size_t)k * nq + t] = df_mul(X[(size_t)k * nq + t], idg[k]);
                    __syncwarp();
                    if (on) {
                        const int r0 = max(0, k - UWe);
                        const float2 xk = X[(size_t)k * nq + t];
                        for (int rr = r0 + rs; rr < k; rr += 4)
                            X[(size_t)rr * nq + t] = df_sub(X[(size_t)rr * nq + t], df_mul(band_at(rr, k), xk));
                    }
                    __syncwarp();
                }
            }
        }
    }
    __syncthreads();
    // S[l, m] = A_bb[l, m] - w(l -> ql) (A_ii^{-1})[ql, qm] w(qm -> m), column-major
    float2 *S = out + Ld.off;
    for (int e = tid; e < r * r; e += nt) {
        const int l = e % r, m = e / r;
        int il, jl, im, jm;
        ring_node_mx(a, bb, l, il, jl);
        ring_node_mx(a, bb, m, im, jm);
        const int dx = im - il, dy = jm - jl;
        float2 v = make_float2(0.f, 0.f);
        if (dx == 0 && dy == 0) v = wr[l * 6 + DIR_C];
        else if (dx == 1 && dy == 0) v = wr[l * 6 + DIR_E];
        else if (dx == -1 && dy == 0) v = wr[l * 6 + DIR_W];
        else if (dx == 0 && dy == 1) v = wr[l * 6 + DIR_N];
        else if (dx == 0 && dy == -1) v = wr[l * 6 + DIR_S];
        if (ni > 0) {
            int il2, jl2, dl, im2, jm2, dm;
            if (inner_nb(a, bb, il, jl, il2, jl2, dl) && inner_nb(a, bb, im, jm, im2, jm2, dm)) {
                const int ql = il2 + ia * jl2, qm = im2 + ia * jm2;
                const float2 x = X[(size_t)ql * nq + inner_id[qm]];
                v = df_sub(v, df_mul(df_mul(wr[l * 6 + dl], x), wr[m * 6 + 5]));
            }
        }
        S[e] = v;
    }
}

cudaError_t mx_leaf(const LeafDesc *d_leaves, const std::vector<LeafDesc> &h_leaves, int max_a, int max_b,
                    const double *b, const double *c, const double *d, float2 *out, Status *st, int stage,
                    cudaStream_t s, KTimer &kt) {
    const size_t smem = mx_leaf_smem_bytes(max_a, max_b);
    cudaError_t e = cudaFuncSetAttribute(k_mx_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    double fl = 0.0;  // the same algorithmic count as the FP64 leaf
    for (const LeafDesc &L : h_leaves) {
        const double ia = L.a - 2, ib = L.b - 2;
        if (ia <= 0 || ib <= 0) continue;
        const double ni = ia * ib, nq = (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
        fl += 4.0 * ni * ia * ia + 6.0 * nq * ni * ia;
    }
    kt.begin(GM_K_LEAF, fl, s);
    k_mx_leaf<<<(int)h_leaves.size(), LEAF_THREADS, smem, s>>>(d_leaves, b, c, d, out, st, stage);
    kt.end(s);
    return cudaGetLastError();
}

}  // namespace gm
