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
#include "smem_limit.h"

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

// ----------------------------------------------------------------------------- by lines

// The same S by block elimination of the interior one grid line at a time (lines
// jj = 0 .. ib - 1 of ia unknowns each; A_ii is block tridiagonal in this order, with
// diagonal couplings between neighbouring lines).  With the lines below jj eliminated,
// the state is
//   Sig : the Schur complement on the ring (starts as A_bb),
//   C   : ring -> line jj couplings (r x ia),   C' : line jj -> ring (ia x r),
//   T   : the line's block (ia x ia),           N  : line jj -> line jj + 1 (diagonal),
// and eliminating line jj is
//   [P | Q] = T^{-1} [C' | N]       (Gauss-Jordan with partial pivoting within the line)
//   Sig    -= C P
//   T'      = D_{jj+1} - S_{jj+1} Q,   C_next = direct - C Q,   C'_next = direct - S_{jj+1} P
// (S_{jj+1}: line jj + 1 -> line jj, diagonal).  Fourteen block steps for a 16 x 16 leaf
// instead of 196 scalar ones, and about a third of the band kernel's shared memory, so
// several leaves share an SM.  Pivoting stays within a line (like the blocked sweep's
// block-local pivoting): a pivot far below the line's diagonal scale raises the growth
// flag, and the automatic mode then rebuilds the problem in FP64.
//
// Only ring nodes whose interior neighbour lies in an eliminated line (or the current
// one) couple to the state; they are listed in line order (tl), so the ones in play
// after line jj are a prefix of the list.

constexpr int LINE_THREADS = 256;

size_t mx_leaf_lines_smem_bytes(int a, int b) {
    const int ia = a - 2, ib = b - 2, r = 2 * a + 2 * b - 4;
    const int ni = (ia > 0 && ib > 0) ? ia * ib : 0;
    const int WM = (2 * ia + r) | 1, CS = ia | 1;
    return 8 * ((size_t)r * r + 2 * (size_t)ia * WM + 2 * (size_t)r * CS + (size_t)ni * 5 + 2 * (size_t)r +
                (size_t)ia) +
           4 * (3 * (size_t)r + 2 * (size_t)ia) + 16;
}

// df32 a + b with an error of a few units of 2^-48 max(|a|, |b|) (df_add also keeps it
// relative to |a + b| under cancellation); enough for these sums, at half the instructions
__device__ __forceinline__ float2 df_add_quick(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    return fast_two_sum(s.x, s.y + (a.y + b.y));
}

__global__ void __launch_bounds__(LINE_THREADS)
k_mx_leaf_lines(const LeafDesc *__restrict__ leaves, const double *__restrict__ bf0, const double *__restrict__ cf0,
                const double *__restrict__ df0, float2 *__restrict__ out, Status *st, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LeafDesc Ld = leaves[blockIdx.x];
    const int n = Ld.n;
    const double *bf = bf0 + Ld.coef, *cf = cf0 + Ld.coef, *df = df0 + Ld.coef;
    const int a = Ld.a, bb = Ld.b, ia = a - 2, ib = bb - 2, r = 2 * a + 2 * bb - 4;
    // row strides in float2, odd so that a column read across rows spreads over the banks
    const int WM = (2 * ia + r) | 1;  // row of M: [T | C' (by ring position) | N | pad]
    const int CS = ia | 1;            // row of C
    const double ih = n + 1.0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    float2 *Sig = (float2 *)smem_raw;            // r x r, column-major
    float2 *Mb = Sig + (size_t)r * r;            // 2 x ia x WM
    float2 *Cb = Mb + 2 * (size_t)ia * WM;       // 2 x r x CS
    float2 *wint = Cb + 2 * (size_t)r * CS;      // ni x 5: C, E, W, N, S of each interior equation
    float2 *wdir = wint + (size_t)ia * ib * 5;   // r: ring node -> its interior neighbour
    float2 *wbak = wdir + r;                     // r: interior neighbour -> ring node
    float2 *pvs = wbak + r;                      // ia: pivots of the current line
    int *tl = (int *)(pvs + ia);                 // r: ring nodes with an interior neighbour, by line
    int *iln = tl + r;                           // r: line of the interior neighbour (-1: corner)
    int *iix = iln + r;                          // r: its position in the line
    int *prow = iix + r;                         // ia: pivot row of each column of T
    auto gnode = [&](int ii, int jj) { return (Ld.x0 + 1 + ii) + n * (Ld.y0 + 1 + jj); };
    // listed ring nodes in play once lines 0 .. jj are in: the bottom row and the side
    // nodes of each line, the top row with the last line
    auto in_play = [&](int jj) { return (a - 2) + 2 * (jj + 1) + (jj == ib - 1 ? a - 2 : 0); };

    // weights (FP64 stencil, then df32) and the ring's bookkeeping
    for (int q = tid; q < ia * ib; q += LINE_THREADS) {
        const int g = gnode(q % ia, q / ia);
#pragma unroll
        for (int dir = 0; dir < 5; ++dir) wint[q * 5 + dir] = df_from_d(stencil_w_mx(bf, cf, df, ih, g, dir));
    }
    for (int e = tid; e < r * r; e += LINE_THREADS) Sig[e] = make_float2(0.f, 0.f);
    for (int l = tid; l < r; l += LINE_THREADS) {
        int il, jl, ii, jj, dir;
        ring_node_mx(a, bb, l, il, jl);
        const int gl = (Ld.x0 + il) + n * (Ld.y0 + jl);
        if (inner_nb(a, bb, il, jl, ii, jj, dir)) {
            iln[l] = jj;
            iix[l] = ii;
            wdir[l] = df_from_d(stencil_w_mx(bf, cf, df, ih, gl, dir));
            wbak[l] = df_from_d(stencil_w_mx(bf, cf, df, ih, gnode(ii, jj), opposite(dir)));
        } else {
            iln[l] = -1;
            iix[l] = -1;
        }
        // the list: bottom row, then (left, right) of each line, then the top row
        const int nb_ = a - 2;
        if (l < nb_) tl[l] = 1 + l;
        else if (l < nb_ + 2 * ib) {
            const int j2 = (l - nb_) >> 1;
            tl[l] = ((l - nb_) & 1) ? a + j2 : r - 1 - j2;
        } else if (l < 2 * nb_ + 2 * ib) {
            tl[l] = 2 * a + bb - 4 - (l - nb_ - 2 * ib);
        }
    }
    __syncthreads();
    // A_bb: each ring node's own weight and its weights on ring neighbours
    for (int l = tid; l < r; l += LINE_THREADS) {
        int il, jl;
        ring_node_mx(a, bb, l, il, jl);
        const int gl = (Ld.x0 + il) + n * (Ld.y0 + jl);
        Sig[l + (size_t)r * l] = df_from_d(stencil_w_mx(bf, cf, df, ih, gl, DIR_C));
        const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1}, dd[4] = {DIR_E, DIR_W, DIR_N, DIR_S};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i2 = il + dx[q], j2 = jl + dy[q];
            if (i2 < 0 || i2 >= a || j2 < 0 || j2 >= bb) continue;
            if (!(i2 == 0 || i2 == a - 1 || j2 == 0 || j2 == bb - 1)) continue;  // interior
            int m;
            if (j2 == 0) m = i2;
            else if (i2 == a - 1) m = a - 1 + j2;
            else if (j2 == bb - 1) m = (a - 1) + (bb - 1) + (a - 1 - i2);
            else m = 2 * (a - 1) + (bb - 1) + (bb - 1 - j2);
            Sig[l + (size_t)r * m] = df_from_d(stencil_w_mx(bf, cf, df, ih, gl, dd[q]));
        }
    }
    float2 *M = Mb, *Mn = Mb + (size_t)ia * WM, *C = Cb, *Cn = Cb + (size_t)r * CS;
    // line 0: M = [D_0 | direct C' | diag N_0], C = direct
    for (int e = tid; e < ia * WM; e += LINE_THREADS) {
        const int k = e / WM, c = e % WM;
        float2 v = make_float2(0.f, 0.f);
        if (c < ia) {
            if (c == k) v = wint[k * 5 + DIR_C];
            else if (c == k + 1) v = wint[k * 5 + DIR_E];
            else if (c == k - 1) v = wint[k * 5 + DIR_W];
        } else if (c < ia + r) {
            const int l = c - ia;
            if (iln[l] == 0 && iix[l] == k) v = wbak[l];
        } else if (c - ia - r == k && ib > 1) {
            v = wint[k * 5 + DIR_N];
        }
        M[e] = v;
    }
    for (int e = tid; e < r * ia; e += LINE_THREADS) {
        const int l = e / ia, k = e % ia;
        C[(size_t)l * CS + k] = (iln[l] == 0 && iix[l] == k) ? wdir[l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // thread roles in the Gauss-Jordan steps: lane -> (row, column offset); rows per pass
    const int RP = ia <= 16 ? 16 : 32, CPW = 32 / RP;
    const int grow_ = lane % RP, gcol = warp * CPW + lane / RP, gstride = 8 * CPW;
    bool grow = false, bad = false;
    float pmin = 3.0e38f;
    for (int jj = 0; jj < ib; ++jj) {
        const int L = in_play(jj);
        const bool more = jj + 1 < ib;
        const int ncn = more ? ia : 0;  // columns of N
        const int nfix = L + ncn;       // columns right of T in play
        // Gauss-Jordan on M without moving rows: column t's pivot row is prow[t]; rows
        // stay unscaled until the end (row p_t holds pivot p_t times solution row t)
        unsigned used = 0u;
        for (int t = 0; t < ia; ++t) {
            // pivot: the unused row of largest |hi| in column t (the lowest among equals);
            // key 0 for used rows and padding lanes, |hi| bits + 1 otherwise (NaN as 0)
            unsigned key = 0u;
            if (lane < ia && !((used >> lane) & 1u)) {
                const float v = fabsf(M[(size_t)lane * WM + t].x);
                key = (v == v ? __float_as_uint(v) : 0u) + 1u;
            }
            const unsigned kmax = __reduce_max_sync(FULL, key);
            const int p = (int)__reduce_min_sync(FULL, key == kmax ? (unsigned)lane : 0xffffffffu);
            used |= 1u << p;
            const float2 pv = M[(size_t)p * WM + t];
            if (tid == 0) {
                prow[t] = p;
                pvs[t] = pv;
                const float ap = fabsf(pv.x);
                if (!(ap > 0.f) || !(ap == ap)) bad = true;
                pmin = fminf(pmin, ap);
                if (ap < 0x1p-12f * fabsf(wint[(t + ia * jj) * 5 + DIR_C].x)) grow = true;
            }
            // every other row: row -= (row[t] / pivot) * pivot row, over the columns in play
            if (grow_ < ia && grow_ != p) {
                const float2 g = df_mul(M[(size_t)grow_ * WM + t], df_rcp(pv));
                float2 *Mr = M + (size_t)grow_ * WM;
                const float2 *Mp = M + (size_t)p * WM;
                const int nT = ia - 1 - t;
                for (int q = gcol; q < nT + nfix; q += gstride) {
                    const int c = q < nT ? t + 1 + q : (q < nT + L ? ia + tl[q - nT] : ia + r + (q - nT - L));
                    Mr[c] = df_sub(Mr[c], df_mul(g, Mp[c]));
                }
            }
            __syncthreads();
        }
        // scale the solution rows: [P | Q] row t = row p_t / pivot t
        for (int e = tid; e < ia * nfix; e += LINE_THREADS) {
            const int t = e / nfix, q = e % nfix;
            const int c = q < L ? ia + tl[q] : ia + r + (q - L);
            float2 &x = M[(size_t)prow[t] * WM + c];
            x = df_mul(x, df_rcp(pvs[t]));
        }
        __syncthreads();
        // Sig -= C P over the ring nodes in play, 2 x 2 entries per thread
        const int L2h = (L + 1) >> 1;
        for (int e = tid; e < L2h * L2h; e += LINE_THREADS) {
            const int i0 = 2 * (e % L2h), j0 = 2 * (e / L2h);
            const int l0 = tl[i0], l1 = i0 + 1 < L ? tl[i0 + 1] : l0;
            const int m0 = tl[j0], m1 = j0 + 1 < L ? tl[j0 + 1] : m0;
            float2 a00 = make_float2(0.f, 0.f), a01 = a00, a10 = a00, a11 = a00;
            for (int t = 0; t < ia; ++t) {
                const float2 c0 = C[(size_t)l0 * CS + t], c1 = C[(size_t)l1 * CS + t];
                const float2 *Pt = M + (size_t)prow[t] * WM + ia;
                const float2 p0 = Pt[m0], p1 = Pt[m1];
                a00 = df_add_quick(a00, df_mul(c0, p0));
                a01 = df_add_quick(a01, df_mul(c0, p1));
                a10 = df_add_quick(a10, df_mul(c1, p0));
                a11 = df_add_quick(a11, df_mul(c1, p1));
            }
            Sig[l0 + (size_t)r * m0] = df_sub(Sig[l0 + (size_t)r * m0], a00);
            if (j0 + 1 < L) Sig[l0 + (size_t)r * m1] = df_sub(Sig[l0 + (size_t)r * m1], a01);
            if (i0 + 1 < L) Sig[l1 + (size_t)r * m0] = df_sub(Sig[l1 + (size_t)r * m0], a10);
            if (i0 + 1 < L && j0 + 1 < L) Sig[l1 + (size_t)r * m1] = df_sub(Sig[l1 + (size_t)r * m1], a11);
        }
        if (more) {
            const int j1 = jj + 1, Ln = in_play(j1);
            // next line's T = D - S Q and its C' = direct - S P, N
            for (int e = tid; e < ia * WM; e += LINE_THREADS) {
                const int k = e / WM, c = e % WM;
                const int q1 = k + ia * j1;  // interior index of row k of the next line
                float2 v = make_float2(0.f, 0.f);
                if (c < ia) {
                    if (c == k) v = wint[q1 * 5 + DIR_C];
                    else if (c == k + 1) v = wint[q1 * 5 + DIR_E];
                    else if (c == k - 1) v = wint[q1 * 5 + DIR_W];
                    v = df_sub(v, df_mul(wint[q1 * 5 + DIR_S], M[(size_t)prow[k] * WM + ia + r + c]));
                } else if (c < ia + r) {
                    const int l = c - ia, li = iln[l];
                    if (li == j1 && iix[l] == k) v = wbak[l];
                    else if (li >= 0 && li <= jj) v = df_neg(df_mul(wint[q1 * 5 + DIR_S], M[(size_t)prow[k] * WM + c]));
                } else if (c - ia - r == k && j1 + 1 < ib) {
                    v = wint[q1 * 5 + DIR_N];
                }
                Mn[e] = v;
            }
            // next C = direct - C Q
            for (int e = tid; e < Ln * ia; e += LINE_THREADS) {
                const int l = tl[e / ia], k = e % ia;
                float2 v = (iln[l] == j1 && iix[l] == k) ? wdir[l] : make_float2(0.f, 0.f);
                if (iln[l] <= jj) {
                    float2 acc = make_float2(0.f, 0.f);
                    for (int t = 0; t < ia; ++t)
                        acc = df_add_quick(acc, df_mul(C[(size_t)l * CS + t], M[(size_t)prow[t] * WM + ia + r + k]));
                    v = df_sub(v, acc);
                }
                Cn[(size_t)l * CS + k] = v;
            }
        }
        __syncthreads();
        float2 *tm = M; M = Mn; Mn = tm;
        float2 *tc = C; C = Cn; Cn = tc;
    }
    if (tid == 0) {
        record_pivot_mx(st + Ld.prob, bad ? 0.0 : (double)pmin, stage);
        if (grow) atomicOr(&st[Ld.prob].growth, 1);
    }
    float2 *S = out + Ld.off;
    for (int e = tid; e < r * r; e += LINE_THREADS) S[e] = Sig[e];
}

cudaError_t mx_leaf(const LeafDesc *d_leaves, const std::vector<LeafDesc> &h_leaves, int max_a, int max_b,
                    const double *b, const double *c, const double *d, float2 *out, Status *st, int stage,
                    cudaStream_t s, KTimer &kt) {
    // by lines when every leaf has an interior and its lines fit one warp's lanes
    bool lines = true;
    for (const LeafDesc &L : h_leaves) lines = lines && L.a >= 3 && L.b >= 3 && L.a - 2 <= 32;
    const size_t smem = lines ? mx_leaf_lines_smem_bytes(max_a, max_b) : mx_leaf_smem_bytes(max_a, max_b);
    cudaError_t e = raise_smem_limit(lines ? (const void *)k_mx_leaf_lines : (const void *)k_mx_leaf, smem);
    if (e != cudaSuccess) return e;
    double fl = 0.0;  // the same algorithmic count as the FP64 leaf
    for (const LeafDesc &L : h_leaves) {
        const double ia = L.a - 2, ib = L.b - 2;
        if (ia <= 0 || ib <= 0) continue;
        const double ni = ia * ib, nq = (ia == 1 || ib == 1) ? ni : 2 * ia + 2 * ib - 4;
        fl += 4.0 * ni * ia * ia + 6.0 * nq * ni * ia;
    }
    kt.begin(GM_K_LEAF, fl, s);
    if (lines)
        k_mx_leaf_lines<<<(int)h_leaves.size(), LINE_THREADS, smem, s>>>(d_leaves, b, c, d, out, st, stage);
    else
        k_mx_leaf<<<(int)h_leaves.size(), LEAF_THREADS, smem, s>>>(d_leaves, b, c, d, out, st, stage);
    kt.end(s);
    return cudaGetLastError();
}

}  // namespace gm
