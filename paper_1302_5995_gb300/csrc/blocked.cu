// Blocked Gauss-Jordan sweep with block-local pivoting for the mixed-precision build.
//
// [M | Z] (double-float, column-major) is reduced 64 columns at a time.  At the step
// with pivot block rows/columns J = [k, k + 64):
//   1. factor : one CTA inverts A11 = W(J, J) in FP32 by Gauss-Jordan with partial
//               pivoting among the rows of J (X0 ~ A11^{-1} to FP32 accuracy); the rows of
//               X0 and of A11 are cut into digit planes.
//   2. slice  : the rows of F = W(i not in J, J) into digit planes (same launch as 3);
//               a row below J whose entry in a column of J exceeds
//               that column's pivot by a large factor raises the growth flag (partial
//               pivoting over all rows would have chosen it).
//   3. R = A11^{-1} A12 by one step of iterative refinement, every product a split
//      product on the tensor cores, one CTA per 64 columns of A12 (fused with step 2):
//               R0 = X0 A12,   E = A12 - A11 R0,   R = R0 + X0 E,
//      R is written into the pivot rows and sliced.
//   4. update : W(i, j) -= (F R)(i, j) for every row i outside J (tensor cores).
// After the last step the right block of W holds M^{-1} Z.  The pivot rows keep the
// same row set as J (pivoting only chooses how A11 is inverted), so no row of W moves.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "blocked.h"
#include "gm_internal.h"
#include "kernels.h"
#include "mixed_dev.cuh"

namespace gm {

constexpr int NBK = BLK_NB;  // 64
constexpr int LDF = NBK + 1;  // padded row length of the df32 shared tiles

// ----------------------------------------------------------------------------- factor

constexpr int FAC_THREADS = 288;  // 256 update threads and the panel warp
// Sort key of a pivot candidate in one 32-bit word, for a single warp max-reduction: the
// top 26 bits are |v| (its float bits with the six lowest cleared; a NaN counts as 0,
// and 64 is added so every unused row beats a used one), the low six bits 63 - row, so
// the lowest row wins among candidates equal to 2^-17 relative.  A used row has key 0.
__device__ __forceinline__ unsigned piv_key(float v, int r, bool used) {
    const float a = fabsf(v);
    const unsigned bits = a == a ? __float_as_uint(a) : 0u;
    return used ? 0u : (((bits & ~63u) + 64u) | (unsigned)(63 - r));
}

// Digit planes of 64 rows x 64 k from a shared tile: thread (row, segment) cuts 16
// consecutive entries of its row (the four segments of a row are consecutive lanes, so
// the row maximum takes two shuffles) and stores them 16 bytes at a time.
template <int S, class Get>
__device__ __forceinline__ void slice_rows64(Get get, int r, int seg, __nv_bfloat16 *__restrict__ dig, int64_t plane,
                                             int64_t r64, int *__restrict__ ex) {
    float2 v[16];
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        v[c] = get(r, seg * 16 + c);
        mx = fmaxf(mx, fabsf(v[c].x));
    }
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    const int e = exp_of_max(mx * 1.0000001f);
    if (seg == 0) ex[r64] = e;
    uint32_t pk[S][8];
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
        float d0[S], d1[S];
        digits<S>(v[c], e, d0);
        digits<S>(v[c + 1], e, d1);
#pragma unroll
        for (int q = 0; q < S; ++q) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(d0[q], d1[q]);
            pk[q][c / 2] = *(const uint32_t *)&h;
        }
    }
#pragma unroll
    for (int q = 0; q < S; ++q) {
        uint4 *dst = (uint4 *)(dig + (int64_t)q * plane + r64 * NBK + seg * 16);
        dst[0] = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
        dst[1] = make_uint4(pk[q][4], pk[q][5], pk[q][6], pk[q][7]);
    }
}

// X0 ~ A11^{-1} by Gauss-Jordan in FP32 with partial pivoting among the rows of the
// block, blocked by panels of 8 pivots, in place.  Rows never move: the pivot of column t
// is the unused row p_t of largest |entry| (the lowest of rows within 2^-17 of it, see
// piv_key).  On [A11 | I] the right-hand column of row p_t changes only from step t on,
// and step t turns column t of the left half into a unit column, so column t's slot holds
// the right-hand column of p_t from then on: at the end slot (r, t) is entry (r, p_t) of
// the right half, and X0(t, i) = slot(p_t, step(i)).
//
// With S_q the 64 x 64 slots after panels 0 .. q - 1, panel q's transform T_q (64 x 8)
// maps S_q to S_{q+1}: with P the panel's 8 pivot rows, new[r] = [r not in P] old[r] +
// sum_u T(r, u) old[p_u] on every slot but the panel's own, which become T's columns (the
// right-hand columns of P, which were unit columns, transform to exactly those).  Column
// u of T starts as the unit vector of p_u when p_u is chosen (no earlier step used that
// row as a source) and then takes the remaining steps' row operations.
//
// The 256 update threads hold the slots in registers (thread (rp, cg): rows 2 rp, 2 rp + 1,
// slots 8 cg .. 8 cg + 7); a ninth warp (the panel warp) holds none and runs one panel
// ahead.  In step k (one block barrier each, k = 0 .. 8):
//   - the panel warp reads panel k's slots of S_{k-1} and the pivot rows of panel k - 1
//     from shared memory, applies T_{k-1} to them itself (the same multiply-adds in the
//     same order as the update threads, so the values are the same), eliminates the
//     64 x 8 panel in registers (two rows per lane, the pivot found by one warp reduction
//     of the packed keys, the pivot row broadcast by shuffles) and publishes T_k;
//   - the update threads apply T_{k-1} (S_{k-1} -> S_k, the pivot rows read from S_{k-1}
//     in shared memory) and store S_k for the next step; in step 0 they cut A11 into
//     its digit planes instead.
// S_q alternates between two shared buffers, T_q between two tables.  The arithmetic is
// Gauss-Jordan on [A11 | I] with the same roundings, less the work on the unit columns.
constexpr int FAC_UPD = 256;  // update threads; the panel warp is warp 8
constexpr int FSL = 68;       // row stride (floats) of the shared slot buffers

template <int S>
__global__ void __launch_bounds__(FAC_THREADS)
k_blk_factor(const SysDesc *__restrict__ sys, const float2 *__restrict__ ws, int k, __nv_bfloat16 *__restrict__ x_dig,
             __nv_bfloat16 *__restrict__ a_dig, int64_t plane, int *__restrict__ x_ex, int *__restrict__ a_ex,
             float *__restrict__ pmag, Status *st, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    float2 *Adf = (float2 *)smem_raw;      // [64][LDF] A11 (df32)
    float *Sb = (float *)(Adf + 64 * LDF);  // two buffers [64][FSL]: S_q in buffer q & 1
    float *Xs = Sb;                         // [64][65] rows of X0, after the last step
    __shared__ float s_pm[64];
    __shared__ float TCs[2][64][9];  // T_q in table q & 1
    __shared__ int Ps[2][8];
    __shared__ int s_step[64], s_prow[64];
    const SysDesc Sy = sys[blockIdx.x];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    const float2 *W = ws + Sy.off;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool upd = tid < FAC_UPD;
    const int rp = upd ? tid >> 3 : 0, cg = tid & 7;  // update thread: rows 2 rp + (0, 1), slots 8 cg + (0 .. 7)
    const unsigned FULL = 0xffffffffu;
    constexpr int BUF = 64 * FSL;
    float a[2][8];
    if (upd) {  // A11, padded with the identity beyond nbe (all loads in flight at once)
        constexpr int NL = 64 * 64 / FAC_UPD;
        float2 v[NL];
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int e = tid + q * FAC_UPD, i = e % 64, j = e / 64;
            v[q] = (i < nbe && j < nbe) ? W[(size_t)(k + j) * m + k + i] : make_float2(i == j ? 1.f : 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int e = tid + q * FAC_UPD;
            Adf[(e % 64) * LDF + e / 64] = v[q];
        }
    }
    __syncthreads();
    if (upd) {  // S_0 = A11 into buffer 0
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int r = 2 * rp + rr;
#pragma unroll
            for (int v = 0; v < 8; ++v) a[rr][v] = Adf[r * LDF + 8 * cg + v].x;
            *(float4 *)&Sb[r * FSL + 8 * cg] = make_float4(a[rr][0], a[rr][1], a[rr][2], a[rr][3]);
            *(float4 *)&Sb[r * FSL + 8 * cg + 4] = make_float4(a[rr][4], a[rr][5], a[rr][6], a[rr][7]);
        }
    }
    __syncthreads();
    // the panel warp's state: T of the last panel for its rows lane and lane + 32, that
    // panel's pivot rows, and which of its rows have been pivots
    float tc[2][8];
    int pidx[8];
    bool used0 = false, used1 = false;
#pragma unroll 1
    for (int kp = 0; kp <= 8; ++kp) {
        const float *Sprev = Sb + (size_t)((kp > 0 ? kp - 1 : 0) & 1) * BUF;  // S_{kp-1} (S_0 at kp = 0)
        if (!upd) {
            if (kp < 8) {
                const int t0 = kp * 8;
                float pv[2][8], pivs[8];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4 x0 = *(const float4 *)&Sprev[(lane + 32 * r) * FSL + t0];
                    const float4 x1 = *(const float4 *)&Sprev[(lane + 32 * r) * FSL + t0 + 4];
                    pv[r][0] = x0.x; pv[r][1] = x0.y; pv[r][2] = x0.z; pv[r][3] = x0.w;
                    pv[r][4] = x1.x; pv[r][5] = x1.y; pv[r][6] = x1.z; pv[r][7] = x1.w;
                }
                if (kp > 0) {  // S_{kp-1} -> S_kp on the panel's slots
                    bool inP0 = false, inP1 = false;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        inP0 |= pidx[u] == lane;
                        inP1 |= pidx[u] == lane + 32;
                    }
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        pv[0][v] = inP0 ? 0.f : pv[0][v];
                        pv[1][v] = inP1 ? 0.f : pv[1][v];
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const float4 q0 = *(const float4 *)&Sprev[pidx[u] * FSL + t0];
                        const float4 q1 = *(const float4 *)&Sprev[pidx[u] * FSL + t0 + 4];
                        const float q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                        for (int r = 0; r < 2; ++r)
#pragma unroll
                            for (int v = 0; v < 8; ++v) pv[r][v] = fmaf(tc[r][u], q[v], pv[r][v]);
                    }
                }
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    tc[0][v] = 0.f;
                    tc[1][v] = 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    // the fast reciprocal of both candidates, ahead of the reduction (the
                    // pivot's comes from its lane): X0 only needs FP32 accuracy (the R step
                    // refines it)
                    const float ip0 = __fdividef(1.0f, pv[0][u]), ip1 = __fdividef(1.0f, pv[1][u]);
                    const unsigned key = __reduce_max_sync(
                        FULL, max(piv_key(pv[0][u], lane, used0), piv_key(pv[1][u], lane + 32, used1)));
                    const int p = 63 - (int)(key & 63u), src = p & 31;
                    const bool mine0 = lane == p, mine1 = lane + 32 == p, hp = p >= 32;
                    used0 |= mine0;
                    used1 |= mine1;
                    tc[0][u] = mine0 ? 1.f : 0.f;
                    tc[1][u] = mine1 ? 1.f : 0.f;
                    float prv[8], prt[8];
#pragma unroll
                    for (int v = u; v < 8; ++v) prv[v] = __shfl_sync(FULL, hp ? pv[1][v] : pv[0][v], src);
#pragma unroll
                    for (int v = 0; v <= u; ++v) prt[v] = __shfl_sync(FULL, hp ? tc[1][v] : tc[0][v], src);
                    const float piv = prv[u], ip = __shfl_sync(FULL, hp ? ip1 : ip0, src);
                    pivs[u] = piv;
                    pidx[u] = p;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const bool isp = r ? mine1 : mine0;
                        const float g = pv[r][u] * ip;
#pragma unroll
                        for (int v = u; v < 8; ++v) pv[r][v] = isp ? prv[v] * ip : fmaf(-g, prv[v], pv[r][v]);
#pragma unroll
                        for (int v = 0; v <= u; ++v) tc[r][v] = isp ? prt[v] * ip : fmaf(-g, prt[v], tc[r][v]);
                    }
                }
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    TCs[kp & 1][lane][v] = tc[0][v];
                    TCs[kp & 1][lane + 32][v] = tc[1][v];
                }
                if (lane < 8) {  // the panel's pivots (lane u: pivot u; compile-time indices)
                    float pm = 0.f;
                    int pi = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (lane == u) {
                            pm = fabsf(pivs[u]);
                            pi = pidx[u];
                        }
                    s_pm[t0 + lane] = pm;
                    if (t0 + lane < nbe) pmag[(size_t)blockIdx.x * 64 + t0 + lane] = pm;
                    Ps[kp & 1][lane] = pi;
                    s_step[pi] = t0 + lane;
                    s_prow[t0 + lane] = pi;
                }
            }
        } else if (kp == 0) {  // while the panel warp takes panel 0: A11's digit planes (K = 64)
            const int row = tid >> 2, seg = tid & 3;
            slice_rows64<S>([&](int r, int c) { return Adf[r * LDF + c]; }, row, seg, a_dig, plane,
                            (int64_t)blockIdx.x * 64 + row, a_ex);
        } else {  // S_{kp-1} -> S_kp on this thread's 2 x 8 slots
            const int tb = (kp - 1) & 1;
            float tcr[2][8];
            int pu[8];
            bool inP[2] = {false, false};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                pu[u] = Ps[tb][u];
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    tcr[rr][u] = TCs[tb][2 * rp + rr][u];
                    inP[rr] |= pu[u] == 2 * rp + rr;
                }
            }
            if (cg == kp - 1) {  // the panel's own slots: T's columns
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                    for (int v = 0; v < 8; ++v) a[rr][v] = tcr[rr][v];
            } else {
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                    for (int v = 0; v < 8; ++v) a[rr][v] = inP[rr] ? 0.f : a[rr][v];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 q0 = *(const float4 *)&Sprev[pu[u] * FSL + 8 * cg];
                    const float4 q1 = *(const float4 *)&Sprev[pu[u] * FSL + 8 * cg + 4];
                    const float q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                        for (int v = 0; v < 8; ++v) a[rr][v] = fmaf(tcr[rr][u], q[v], a[rr][v]);
                }
            }
            if (kp < 8) {
                float *Snew = Sb + (size_t)(kp & 1) * BUF;
#pragma unroll
                for (int rr = 0; rr < 2; ++rr) {
                    const int r = 2 * rp + rr;
                    *(float4 *)&Snew[r * FSL + 8 * cg] = make_float4(a[rr][0], a[rr][1], a[rr][2], a[rr][3]);
                    *(float4 *)&Snew[r * FSL + 8 * cg + 4] = make_float4(a[rr][4], a[rr][5], a[rr][6], a[rr][7]);
                }
            }
        }
        __syncthreads();
    }
    pdl_trigger();  // the R kernel may start launching while this one cuts its digits
    if (upd) {  // X0(step(r), p_c) = slot(r, c)
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int t = s_step[2 * rp + rr];
#pragma unroll
            for (int v = 0; v < 8; ++v) Xs[t * 65 + s_prow[8 * cg + v]] = a[rr][v];
        }
    }
    __syncthreads();
    if (tid == 0) {
        float mn = 3.0e38f;
        for (int t = 0; t < nbe; ++t) mn = fminf(mn, s_pm[t]);
        record_pivot_mx(st + Sy.prob, (double)mn, stage);
    }
    if (!upd) return;
    // digit planes of the rows of X0 (FP32: four digits carry it past its accuracy, and
    // only four are read): thread (row, segment) as in slice_rows64
    const int row = tid >> 2, seg = tid & 3;
    slice_rows64<(S < 4 ? S : 4)>([&](int r, int c) { return make_float2(Xs[r * 65 + c], 0.f); }, row, seg, x_dig,
                                  plane, (int64_t)blockIdx.x * 64 + row, x_ex);
}

size_t blk_factor_smem(int split) {
    (void)split;
    // A11 (df32), then two slot buffers (X0 reuses the first)
    return (size_t)64 * LDF * sizeof(float2) + (size_t)2 * 64 * FSL * sizeof(float);
}

// ----------------------------------------------------------------------------- full-K digit tiles

constexpr int KP64 = 72;  // row stride (bf16) of a full-K digit tile: 64 + 8 keeps fragment loads conflict-free

// Rows r0 .. r0 + nrows - 1 of every digit plane (64 k each) into shared [S][64][KP64] by
// cp.async; rows beyond nrows are zero-filled (their source row is r0, in bounds).
template <int S>
__device__ __forceinline__ void cp_async_digits64(const __nv_bfloat16 *__restrict__ dig, int64_t plane, int r0,
                                                  int nrows, __nv_bfloat16 *sm) {
    for (int e = threadIdx.x; e < S * 64 * 8; e += blockDim.x) {
        const int s = e >> 9, rem = e & 511, row = rem >> 3, c = rem & 7;
        const bool ok = row < nrows;
        const __nv_bfloat16 *src = dig + (int64_t)s * plane + (int64_t)(r0 + (ok ? row : 0)) * NBK + c * 8;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(sm + ((size_t)s * 64 + row) * KP64 + c * 8);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0));
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

// ----------------------------------------------------------------------------- R = A11^{-1} A12

// Warps of the R kernel and of the update: a 2 x 4 grid over the 64 x 64 tile, each warp
// 32 rows x 16 columns (two n8 tiles) -- eight warps keep two per scheduler, so one
// warp's dependent latencies hide behind the other's.
constexpr int W_NT = 2;
constexpr int TILE_THREADS = 32 * 2 * (64 / (8 * W_NT));  // 256

// Column exponents of a 64 x TW df32 shared tile D[t][jj] (every thread takes part: P
// consecutive lanes per column).
template <int TW = 64>
__device__ __forceinline__ void col_exps64(const float2 *D, int *ex) {
    constexpr int P = TILE_THREADS / TW;
    const int jj = threadIdx.x / P, part = threadIdx.x % P;
    float mx = 0.f;
    for (int t = part; t < NBK; t += P) mx = fmaxf(mx, fabsf(D[t * LDF + jj].x));
#pragma unroll
    for (int o = 1; o < P; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (part == 0) ex[jj] = exp_of_max(mx * 1.0000001f);
}

// P = A D for a 64 x TW x 64 product (TW = 32 NT): A by rows from a full-K shared digit
// tile Ak ([S][64][KP64], exponents aex), D a df32 shared tile cut by columns into Bk
// (same layout, exponents exB) before the k-steps, which then run without barriers.
template <int S, int NT>
__device__ __forceinline__ void gemm64_full(const __nv_bfloat16 *Ak, const int *__restrict__ aex, const float2 *D,
                                            const int *exB, __nv_bfloat16 *Bk, float2 res[2][NT][4], int kend) {
    constexpr int TW = 32 * NT;
    const int tid = threadIdx.x, warp = tid >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 8 * NT;
    __syncthreads();  // exB written, the previous product done with Bk
    for (int e = tid; e < TW * 64; e += TILE_THREADS) {
        const int jj = e >> 6, t = e & 63;
        float d[S];
        digits<S>(D[t * LDF + jj], exB[jj], d);
#pragma unroll
        for (int q = 0; q < S; ++q) Bk[((size_t)q * 64 + jj) * KP64 + t] = __float2bfloat16_rn(d[q]);
    }
    __syncthreads();
    float acc[S][2][NT][4];
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[g][mt][nt][c] = 0.f;
#pragma unroll 1
    for (int kk = 0; kk < kend; kk += 16) warp_mma_levels<S, KP64, NT>(Ak + kk, Bk + kk, 64, 64, wm, wn, acc);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                res[mt][nt][c] = combine_levels<S, NT>(acc, mt, nt, c, aex[wm + r] + exB[wn + cl] - 12);
            }
}

// Blocks [0, cb): column tiles ct0 .. ct0 + cb - 1 of TW = 32 NT columns right of the pivot
// block (a launch may take any run of them; NT = 1 when the grid
// is small, so twice as many SMs share the step):
//   R0 = X0 A12,  E = A12 - A11 R0,  R = R0 + X0 E  (one refinement step),
// R written into the pivot rows and cut into column digit planes for the update.
// Blocks [cb, cb + rb): 128 rows each: F = W(i, J) (zero inside J) into row digit planes,
// with the growth check against the block pivots.
template <int S, int NT>
__global__ void __launch_bounds__(TILE_THREADS)
k_blk_rfused(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int cb, int ct0,
             const __nv_bfloat16 *__restrict__ x_dig, const __nv_bfloat16 *__restrict__ a11_dig, int64_t plane,
             const int *__restrict__ x_ex, const int *__restrict__ a11_ex, __nv_bfloat16 *__restrict__ fdig,
             int64_t fplane, int *__restrict__ fex, __nv_bfloat16 *__restrict__ rdig, int64_t cplane,
             int *__restrict__ rex, const float *__restrict__ pmag, Status *__restrict__ st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const SysDesc Sy = sys[blockIdx.y];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    float2 *W = ws + Sy.off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if ((int)blockIdx.x >= cb) {
        // a 128 x 64 tile of F through shared memory: read by rows (coalesced over i; the
        // two halves of the block take columns 0-31 and 32-63), digit planes written by
        // warps along the row (coalesced over t)
        float2 *Ft = (float2 *)smem_raw;  // [128][LDF]
        __shared__ float s_mx[2][128];
        __shared__ int s_ex[128];
        const int r = tid & 127, h = tid >> 7;
        const int i0 = ((int)blockIdx.x - cb) * 128, i = i0 + r;
        const bool live = i < m && !(i >= k && i < k + nbe);
        float mx = 0.f;
        bool grow = false;
        for (int t = h * 32; t < h * 32 + 32; ++t) {
            const float2 v = (live && t < nbe) ? W[(size_t)(k + t) * m + i] : make_float2(0.f, 0.f);
            Ft[r * LDF + t] = v;
            const float av = fabsf(v.x);
            mx = fmaxf(mx, av);
            if (t < nbe && i >= k + nbe && av > 16.f * pmag[(size_t)blockIdx.y * 64 + t]) grow = true;
        }
        if (grow) atomicOr(&st[Sy.prob].growth, 1);
        s_mx[h][r] = mx;
        __syncthreads();
        if (h == 0) {
            const int e = exp_of_max(fmaxf(mx, s_mx[1][r]) * 1.0000001f);
            s_ex[r] = e;
            if (i < m) fex[Sy.roff + i] = e;
        }
        __syncthreads();
        for (int rr = warp; rr < 128 && i0 + rr < m; rr += TILE_THREADS / 32) {
            const int64_t row = Sy.roff + i0 + rr;
            const int er = s_ex[rr];
            for (int t = lane; t < NBK; t += 32) {
                float d[S];
                digits<S>(Ft[rr * LDF + t], er, d);
#pragma unroll
                for (int q = 0; q < S; ++q) fdig[(int64_t)q * fplane + row * NBK + t] = __float2bfloat16_rn(d[q]);
            }
        }
        return;
    }
    constexpr int TW = 32 * NT;
    const int j0 = k + nbe + (ct0 + (int)blockIdx.x) * TW;
    if (j0 >= Sy.ncol) return;
    constexpr int SX = S < 4 ? S : 4;
    __nv_bfloat16 *Xk = (__nv_bfloat16 *)smem_raw;  // [SX][64][KP64]: rows of X0
    __nv_bfloat16 *A11k = Xk + SX * 64 * KP64;      // [S][64][KP64]: rows of A11
    __nv_bfloat16 *Bk = A11k + S * 64 * KP64;       // [S][64][KP64]: columns of the right operand
    float2 *Ad = (float2 *)(Bk + S * 64 * KP64);   // [64][LDF]: A12, then E
    float2 *Rd = Ad + 64 * LDF;                     // [64][LDF]: R0, then R
    __shared__ int exB[64];
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 8 * NT;
    const __nv_bfloat16 *xd = x_dig + (int64_t)blockIdx.y * 64 * NBK, *ad = a11_dig + (int64_t)blockIdx.y * 64 * NBK;
    const int *xe = x_ex + blockIdx.y * 64, *ae = a11_ex + blockIdx.y * 64;
    // both left operands (all 64 k) in flight while A12 is read
    cp_async_digits64<SX>(xd, plane, 0, 64, Xk);
    cp_async_digits64<S>(ad, plane, 0, 64, A11k);
    {  // A12 (all loads in flight at once)
        constexpr int NL = TW * 64 / TILE_THREADS;
        float2 v[NL];
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int e = tid + q * TILE_THREADS, t = e & 63, j = j0 + (e >> 6);
            v[q] = (t < nbe && j < Sy.ncol) ? W[(size_t)j * m + k + t] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int e = tid + q * TILE_THREADS;
            Ad[(e & 63) * LDF + (e >> 6)] = v[q];
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();
    col_exps64<TW>(Ad, exB);
    __shared__ int cmax[64], rmax[64];  // column maxima of |X0 E| and |R| (float bits, >= 0)
    if (tid < 64) cmax[tid] = rmax[tid] = 0;
    // three dependent products through one (rolled) copy of the split-product body:
    //   pass 0: R0 = X0 A12 -> Rd;  pass 1: E = A12 - A11 R0 -> Ad;  pass 2: R = R0 + X0 E
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
        float2 res[2][NT][4];
        // K = nbe: the operands are zero beyond the block's live columns.  Passes 0 and 2
        // multiply by the FP32 inverse X0, which four 7-bit digits carry to 2^-28 of each
        // row's maximum -- beyond X0's own accuracy; R0 only has to be good to about FP32
        // (the refinement corrects it) and X0 E is a correction of relative size rho, so
        // four digits of the right operand suffice there.  E itself (pass 1) is a
        // difference of nearly equal terms: full digits.
        if (pass == 1)
            gemm64_full<S, NT>(A11k, ae, Rd, exB, Bk, res, (nbe + 15) & ~15);
        else
            gemm64_full<SX, NT>(Xk, xe, Ad, exB, Bk, res, (nbe + 15) & ~15);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    int r, cl;
                    acc_pos(mt, nt, c, r, cl);
                    const int t = wm + r, jj = wn + cl, j = j0 + jj;
                    if (pass == 0) {
                        Rd[t * LDF + jj] = (t < nbe) ? res[mt][nt][c] : make_float2(0.f, 0.f);
                    } else if (pass == 1) {
                        float2 *q = Ad + t * LDF + jj;
                        *q = (t < nbe) ? df_sub(*q, res[mt][nt][c]) : make_float2(0.f, 0.f);
                    } else {
                        const float2 v = (t < nbe) ? df_add(Rd[t * LDF + jj], res[mt][nt][c]) : make_float2(0.f, 0.f);
                        Rd[t * LDF + jj] = v;
                        if (t < nbe && j < Sy.ncol) {
                            W[(size_t)j * m + k + t] = v;
                            atomicMax(&cmax[jj], __float_as_int(fabsf(res[mt][nt][c].x)));
                            atomicMax(&rmax[jj], __float_as_int(fabsf(v.x)));
                        }
                    }
                }
        if (pass < 2) {
            __syncthreads();
            col_exps64<TW>(pass == 0 ? Rd : Ad, exB);  // column scales of the next product's right operand
        }
    }
    __syncthreads();
    // The refinement step leaves an error of about rho^2 |R|, where rho = |X0 E| / |R| is
    // its contraction factor (kappa(A11) times the FP32 accuracy of X0); the largest rho
    // of the build is reported, and the host decides whether the build is accurate enough.
    if (tid < TW && j0 + tid < Sy.ncol) {
        const float cm = __int_as_float(cmax[tid]), rm = __int_as_float(rmax[tid]);
        if (cm > 0.f) {
            const float rho = rm > 0.f ? cm / rm : __int_as_float(0x7f800000);
            atomicMax(&st[Sy.prob].rho, __float_as_uint(rho));
        }
    }
    col_exps64<TW>(Rd, exB);
    __syncthreads();
    for (int e = tid; e < TW * 64; e += TILE_THREADS) {  // column digit planes of R
        const int jj = e >> 6, t = e & 63, j = j0 + jj;
        if (j >= Sy.ncol) continue;
        const int64_t row = Sy.coff + j;
        if (t == 0) rex[row] = exB[jj];
        float d[S];
        digits<S>(Rd[t * LDF + jj], exB[jj], d);
#pragma unroll
        for (int q = 0; q < S; ++q) rdig[(int64_t)q * cplane + row * NBK + t] = __float2bfloat16_rn(d[q]);
    }
}

size_t blk_rgemm_smem(int split) {
    // R part: three full-K digit tiles (X0 with at most four planes) and two df32 tiles;
    // F part: one 128-row df32 tile
    const size_t sx = split < 4 ? split : 4;
    return std::max((sx + 2 * (size_t)split) * 64 * KP64 * 2 + 2 * 64 * LDF * sizeof(float2),
                    (size_t)128 * LDF * sizeof(float2));
}

// ----------------------------------------------------------------------------- update

// row stride (float2) of the shared copy of a W tile: 66 keeps the epilogue's reads
// (eight rows x four column pairs per half warp) free of bank conflicts
constexpr int WLD = 66;

size_t blk_update_smem(int split) {
    return 2 * (size_t)split * 64 * KP64 * sizeof(__nv_bfloat16) + (size_t)64 * WLD * sizeof(float2);
}

// Which tiles of the update a launch covers.  Tile (ti, tj) holds rows 64 ti .. and the
// columns 64 tj .. right of J.  The look-ahead splits the update in two:
//   UPD_NEXT : column tile 0 (the next block's columns) for every row tile, then the next
//              block's row tile (rows k + 64 ..) for column tiles 1 .. : grid.x = nrt + (column
//              tiles - 1), everything the next factor and R kernel read;
//   UPD_REST : every other tile, grid (nrt, column tiles - 1).
//   (the early-factor schedule of blk_gj_sweep, below:)
//   UPD_A11  : the next pivot block's diagonal tile only (band, 0): the next factor's input;
//   UPD_D2   : the diagonal tile two blocks ahead (band + 1, 1), left out of UPD_REST2;
//   UPD_NEXT2: UPD_NEXT without the tile UPD_A11 takes;
//   UPD_REST2: UPD_REST without the tile UPD_D2 takes.
enum { UPD_ALL = 0, UPD_NEXT = 1, UPD_REST = 2, UPD_A11 = 3, UPD_D2 = 4, UPD_NEXT2 = 5, UPD_REST2 = 6 };

// W(i, j) -= (F R)(i, j) for a 64 x 64 tile of rows outside J: both digit tiles (K = 64)
// and the tile of W arrive by cp.async, then four k-steps of split products without
// barriers, and the epilogue reads W from shared memory (no memory latency after the
// products).
template <int S>
__global__ void __launch_bounds__(TILE_THREADS)
k_blk_update(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int mode, int nrt,
             const __nv_bfloat16 *__restrict__ fdig, int64_t fplane, const int *__restrict__ fex,
             const __nv_bfloat16 *__restrict__ rdig, int64_t rplane, const int *__restrict__ rex) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();  // the next block's factor (one CTA per system) may launch and wait
    __nv_bfloat16 *As = (__nv_bfloat16 *)smem_raw;  // [S][64][KP64]
    __nv_bfloat16 *Bs = As + S * 64 * KP64;
    const SysDesc Sy = sys[blockIdx.z];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    int ti = blockIdx.x, tj = blockIdx.y;
    const int band = k / NBK + 1;  // row tile of the next pivot block
    if (mode == UPD_NEXT || mode == UPD_NEXT2) {
        if (ti >= nrt) {
            tj = ti - nrt + 1;
            ti = band;
        } else if (mode == UPD_NEXT2 && ti == band) {
            return;  // the next pivot block: updated on the chain (UPD_A11)
        }
    } else if (mode == UPD_REST) {
        if (ti == band) return;
        ++tj;
    } else if (mode == UPD_A11) {
        ti = band;
        tj = 0;
    } else if (mode == UPD_D2) {
        ti = band + 1;
        tj = 1;
    }
    const int i0 = ti * 64, j0 = k + nbe + tj * 64;
    if (i0 >= m || j0 >= Sy.ncol) return;
    float2 *W = ws + Sy.off;
    float2 *Wt = (float2 *)(Bs + S * 64 * KP64);  // [64][WLD]: this tile of W, by columns
    __shared__ int s_fe[64], s_re[64];
    cp_async_digits64<S>(fdig + (int64_t)Sy.roff * NBK, fplane, i0, min(64, m - i0), As);
    cp_async_digits64<S>(rdig + (int64_t)Sy.coff * NBK, rplane, j0, min(64, Sy.ncol - j0), Bs);
    // the tile of W itself is only read by the epilogue: its copy overlaps the products
    for (int e = threadIdx.x; e < 64 * 64; e += TILE_THREADS) {
        const int jj = e >> 6, ii = e & 63, i = i0 + ii, j = j0 + jj;
        const bool ok = i < m && j < Sy.ncol;
        const float2 *src = W + (ok ? (size_t)j * m + i : 0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(Wt + jj * WLD + ii);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0));
    }
    asm volatile("cp.async.commit_group;\n" ::);
    if (threadIdx.x < 64) {
        const int i = i0 + threadIdx.x;
        s_fe[threadIdx.x] = i < m ? fex[Sy.roff + i] : 0;
    } else if (threadIdx.x < 128) {
        const int j = j0 + threadIdx.x - 64;
        s_re[threadIdx.x - 64] = j < Sy.ncol ? rex[Sy.coff + j] : 0;
    }
    asm volatile("cp.async.wait_group 1;\n" ::);  // both digit tiles
    __syncthreads();
    const int warp = threadIdx.x >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 8 * W_NT;
    float acc[S][2][W_NT][4];
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < W_NT; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[g][mt][nt][c] = 0.f;
#pragma unroll 1
    for (int kk = 0; kk < nbe; kk += 16) warp_mma_levels<S, KP64, W_NT>(As + kk, Bs + kk, 64, 64, wm, wn, acc);
    asm volatile("cp.async.wait_group 0;\n" ::);  // the tile of W
    __syncthreads();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < W_NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                const int ii = wm + r, jj = wn + cl, i = i0 + ii, j = j0 + jj;
                if (i >= m || j >= Sy.ncol || (i >= k && i < k + nbe)) continue;
                W[(size_t)j * m + i] =
                    df_sub(Wt[jj * WLD + ii], combine_levels<S, W_NT>(acc, mt, nt, c, s_fe[ii] + s_re[jj] - 12));
            }
}

// ----------------------------------------------------------------------------- update, tcgen05

// The same update W(i, j) -= (F R)(i, j) on the fifth-generation tensor cores: a CTA takes
// 128 rows x 64 columns; the digit tiles of F and R (all 64 k) arrive by cp.async in the
// K-major, unswizzled core-matrix layout (8 rows x 16 bytes per core matrix, cores 128
// bytes apart along k and 1024 bytes apart along the rows), one thread issues the
// 21 digit-pair products of each 16-k step as tcgen05.mma (M = 128, N = 64, K = 16,
// bf16 x bf16 -> fp32) into six level accumulators in tensor memory (64 columns each),
// and eight warps read them back (tcgen05.ld) for the same exact level combination and
// double-float subtraction as the mma.sync kernel.  Modes: UPD_ALL, or UPD_REST (the
// look-ahead's rest: column tiles 1 .., the next pivot band's rows left out).
constexpr int TC_ROWS = 128, TC_COLS = 64, TC_TMEM_COLS = 512;

size_t blk_update_tc_smem(int split) {
    return (size_t)split * (TC_ROWS + TC_COLS) * NBK * sizeof(__nv_bfloat16) + 1024;  // + alignment slack
}

// rows r0 .. r0 + R - 1 (zero beyond nrows) of every digit plane (64 k) into the core-matrix
// layout: plane q at q * R * 128 bytes, 16-byte chunk (row, c) at (row / 8) 1024 + c 128 + (row % 8) 16
template <int S, int R, int NT = TILE_THREADS>
__device__ __forceinline__ void cp_async_digits_umma(const __nv_bfloat16 *__restrict__ dig, int64_t plane, int r0,
                                                     int nrows, unsigned char *sm) {
    for (int e = threadIdx.x; e < S * R * 8; e += NT) {
        const int c = e & 7, row = (e >> 3) % R, q = e / (8 * R);
        const bool ok = row < nrows;
        const __nv_bfloat16 *src = dig + (int64_t)q * plane + (int64_t)(r0 + (ok ? row : 0)) * NBK + c * 8;
        const uint32_t dst = smem_u32(sm + (size_t)q * R * 128 + (row >> 3) * 1024 + c * 128 + (row & 7) * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0));
    }
}

template <int S>
__global__ void __launch_bounds__(TILE_THREADS)
k_blk_update_tc(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int mode,
                const __nv_bfloat16 *__restrict__ fdig, int64_t fplane, const int *__restrict__ fex,
                const __nv_bfloat16 *__restrict__ rdig, int64_t rplane, const int *__restrict__ rex,
                Status *__restrict__ st, int limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Fs = base;                                  // S x 16 KB
    unsigned char *Rs = base + (size_t)S * TC_ROWS * 128;      // S x 8 KB
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fe[TC_ROWS], s_re[TC_COLS];
    __shared__ int s_ok;
    const SysDesc Sy = sys[blockIdx.z];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    const bool rest = mode == UPD_REST || mode == UPD_REST2;
    const int i0 = blockIdx.x * TC_ROWS, j0 = k + nbe + (blockIdx.y + (rest ? 1 : 0)) * TC_COLS;
    if (i0 >= m || j0 >= Sy.ncol) return;
    // rows this tile leaves alone: the pivot rows, and in UPD_REST the next pivot band
    const int skip_lo = k, skip_hi = rest ? min(m, k + 2 * NBK) : k + nbe;
    // UPD_REST2, column tile 1: the diagonal tile two blocks ahead is UPD_D2's
    const bool dtile = mode == UPD_REST2 && j0 == k + nbe + TC_COLS;
    if (i0 >= skip_lo && i0 + TC_ROWS <= skip_hi) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2 *W = ws + Sy.off;
    cp_async_digits_umma<S, TC_ROWS>(fdig + (int64_t)Sy.roff * NBK, fplane, i0, min(TC_ROWS, m - i0), Fs);
    cp_async_digits_umma<S, TC_COLS>(rdig + (int64_t)Sy.coff * NBK, rplane, j0, min(TC_COLS, Sy.ncol - j0), Rs);
    asm volatile("cp.async.commit_group;\n" ::);
    if (tid < TC_ROWS) {
        const int i = i0 + tid;
        s_fe[tid] = i < m ? fex[Sy.roff + i] : 0;
    } else if (tid < TC_ROWS + TC_COLS) {
        const int j = j0 + tid - TC_ROWS;
        s_re[tid - TC_ROWS] = j < Sy.ncol ? rex[Sy.coff + j] : 0;
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("cp.async.wait_all;\n" ::);
    asm volatile("fence.proxy.async.shared::cta;\n" ::);  // the copies, visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        constexpr uint32_t idesc = umma_idesc_bf16(TC_ROWS, TC_COLS);
        const int nk = (nbe + 15) >> 4;
        for (int kc = 0; kc < nk; ++kc)
#pragma unroll
            for (int a = 0; a < S; ++a)
#pragma unroll
                for (int b = 0; b < S - a; ++b) {
                    const uint64_t da = umma_desc(smem_u32(Fs + (size_t)a * TC_ROWS * 128 + kc * 256), 128, 1024);
                    const uint64_t db = umma_desc(smem_u32(Rs + (size_t)b * TC_COLS * 128 + kc * 256), 128, 1024);
                    const uint32_t dt = tmem + (uint32_t)((a + b) * TC_COLS);
                    const uint32_t acc = (kc > 0 || a > 0) ? 1u : 0u;  // level a + b starts at (0, a + b)
                    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                 ::"r"(dt), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(&mbar)));
    }
    // this thread's row and 32 columns; their W values are read while the products run
    const int q = warp & 3, h = warp >> 2;
    const int row = 32 * q + lane, i = i0 + row;
    const bool live = i < m && !(i >= skip_lo && i < skip_hi) && !(dtile && i >= k + 2 * NBK && i < k + 3 * NBK);
    float2 w[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const int j = j0 + 32 * h + c;
        w[c] = (live && j < Sy.ncol) ? W[(size_t)j * m + i] : make_float2(0.f, 0.f);
    }
    const bool done = mbar_wait_bounded(&mbar, 0, limit);
    if (tid == 0) s_ok = 1;
    __syncthreads();
    if (!done) {
        s_ok = 0;
        if (lane == 0 && atomicCAS(&st[Sy.prob].code, 0, GM_ETIMEOUT) == 0) st[Sy.prob].where = -1;
    }
    __syncthreads();
    // gave up: the products already issued still write this CTA's tensor memory; wait
    // (bounded) for their commit before the memory is released below
    if (!s_ok && tid == 0) mbar_wait_bounded(&mbar, 0, DRAIN_POLLS);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (s_ok) {
        const int fe = s_fe[row];
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 8) {
            uint32_t v[S][8];
#pragma unroll
            for (int g = 0; g < S; ++g) {
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * TC_COLS + 32 * h + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                             : "=r"(v[g][0]), "=r"(v[g][1]), "=r"(v[g][2]), "=r"(v[g][3]), "=r"(v[g][4]),
                               "=r"(v[g][5]), "=r"(v[g][6]), "=r"(v[g][7])
                             : "r"(ta));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int jj = 32 * h + c0 + c, j = j0 + jj;
                if (!live || j >= Sy.ncol) continue;
                float2 x = make_float2(__uint_as_float(v[S - 1][c]) * pow2f(-7 * (S - 1)), 0.f);
#pragma unroll
                for (int g = S - 2; g >= 0; --g) x = df_add_f(x, __uint_as_float(v[g][c]) * pow2f(-7 * g));
                W[(size_t)j * m + i] = df_sub(w[c0 + c], df_scale(x, fe + s_re[jj] - 12));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ----------------------------------------------------------------------------- update, pipelined tcgen05

// The same update with a CTA per 128-row band and a run of its 64-column tiles.  The
// band's F digits are copied once and stay in shared memory; three copy warps bring the R
// digits of the next tile into the other of two stages while the current tile's 21 x 4
// products run (one thread of a ninth warp, which holds the tensor memory, issues them
// into six level accumulators).  Eight warps finish a tile in two halves: right after its
// products they read the levels back and combine them (the tensor memory is then free for
// the next tile's products), and while the next tile's products run they read that tile
// of W, subtract and store it.  One barrier per tile: after it, the stage and the
// accumulators a tile reuses were last read by work that finished before it.  (An
// M = 128 instruction with N = 64 costs about as many cycles as one with N = 32, so the
// wider tile halves the issue time per column.)
constexpr int TP_COLS = 64, TP_STAGES = 2, TP_THREADS = 384;
constexpr int TP_LOADER = 288;  // first thread of the three copy warps

size_t blk_update_tp_smem(int split) {
    return (size_t)split * (TC_ROWS + TP_STAGES * TP_COLS) * NBK * sizeof(__nv_bfloat16) + 1024;
}

template <int S>
__global__ void __launch_bounds__(TP_THREADS, 1)
k_blk_update_tp(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int mode, int tpc,
                const __nv_bfloat16 *__restrict__ fdig, int64_t fplane, const int *__restrict__ fex,
                const __nv_bfloat16 *__restrict__ rdig, int64_t rplane, const int *__restrict__ rex,
                Status *__restrict__ st, int limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Fs = base;                              // S x 16 KB
    unsigned char *Rs = base + (size_t)S * TC_ROWS * 128;  // TP_STAGES x S x 8 KB
    constexpr int RSTAGE = S * TP_COLS * 128;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fe[TC_ROWS], s_re[TP_STAGES][TP_COLS];
    __shared__ int s_ok;
    const SysDesc Sy = sys[blockIdx.z];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    const bool rest = mode == UPD_REST || mode == UPD_REST2;
    const int i0 = blockIdx.x * TC_ROWS;
    // columns from jb on (UPD_REST: the first 64 are the look-ahead's); rows skip_lo ..
    // skip_hi - 1 are left alone (the pivot rows; in UPD_REST the next pivot band too)
    const int jb = k + nbe + (rest ? 64 : 0);
    const int skip_lo = k, skip_hi = rest ? min(m, k + 2 * NBK) : k + nbe;
    if (i0 >= m || (i0 >= skip_lo && i0 + TC_ROWS <= skip_hi)) return;
    const int ntile = (Sy.ncol - jb + TP_COLS - 1) / TP_COLS, t0 = blockIdx.y * tpc;
    const int nmine = min(tpc, ntile - t0);
    if (nmine <= 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2 *W = ws + Sy.off;
    const __nv_bfloat16 *rd = rdig + (int64_t)Sy.coff * NBK;
    const int *re = rex + Sy.coff;
    auto tile_j0 = [&](int t) { return jb + (t0 + t) * TP_COLS; };
    // R digits of tile t into its stage: by the copy warps (9-11) inside the loop, by all
    // threads before it
    auto load_r = [&](int t, int first, int nthreads) {
        const int j0 = tile_j0(t), sg = t % TP_STAGES, nrows = min(TP_COLS, Sy.ncol - j0);
        unsigned char *sm = Rs + sg * RSTAGE;
        for (int e = tid - first; e < S * TP_COLS * 8; e += nthreads) {
            const int c = e & 7, r = (e >> 3) % TP_COLS, pl = e / (8 * TP_COLS);
            const bool ok = r < nrows;
            const __nv_bfloat16 *src = rd + (int64_t)pl * rplane + (int64_t)(j0 + (ok ? r : 0)) * NBK + c * 8;
            const uint32_t dst = smem_u32(sm + (size_t)pl * TP_COLS * 128 + (r >> 3) * 1024 + c * 128 + (r & 7) * 16);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0));
        }
        if (warp == 9) {  // the exponents of the tile's columns
#pragma unroll
            for (int h2 = 0; h2 < TP_COLS; h2 += 32) {
                const int j = j0 + h2 + lane;
                const bool ok = j < Sy.ncol;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_u32(&s_re[sg][h2 + lane])),
                             "l"(re + (ok ? j : 0)), "r"(ok ? 4 : 0));
            }
        }
    };
    cp_async_digits_umma<S, TC_ROWS, TP_THREADS>(fdig + (int64_t)Sy.roff * NBK, fplane, i0, min(TC_ROWS, m - i0), Fs);
    load_r(0, 0, TP_THREADS);
    asm volatile("cp.async.commit_group;\n" ::);
    if (tid < TC_ROWS) {
        const int i = i0 + tid;
        s_fe[tid] = i < m ? fex[Sy.roff + i] : 0;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
        s_ok = 1;
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    // epilogue warps 0-7: tensor-memory lanes 32 (warp % 4) .., columns 32 (warp / 4) ..
    const int q = warp & 3, h = (warp >> 2) & 1;
    const int row = 32 * q + lane, i = i0 + row;
    const bool row_live = warp < 8 && i < m && !(i >= skip_lo && i < skip_hi);
    float2 acc[32];          // F R of the tile being finished (scaled)
    int pj0 = 0;             // its first column
    bool plive = false;      // this thread's row is written in it
    uint32_t tmem = 0;
    int last = -1;  // the last tile whose products were issued (issuing thread)
    for (int t = 0; t <= nmine; ++t) {
        asm volatile("cp.async.wait_group 0;\n" ::);           // R digits of tile t (and F)
        asm volatile("fence.proxy.async.shared::cta;\n" ::);  // visible to the tensor cores
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        if (t == 0) tmem = s_tmem;
        if (!s_ok) break;
        if (t < nmine && tid == 256) {
            constexpr uint32_t idesc = umma_idesc_bf16(TC_ROWS, TP_COLS);
            const unsigned char *Rb = Rs + (t % TP_STAGES) * RSTAGE;
            const int nk = (nbe + 15) >> 4;
            for (int kc = 0; kc < nk; ++kc)
#pragma unroll
                for (int a = 0; a < S; ++a)
#pragma unroll
                    for (int b = 0; b < S - a; ++b)
                        umma_bf16(tmem + (uint32_t)((a + b) * TP_COLS),
                                  umma_desc(smem_u32(Fs + (size_t)a * TC_ROWS * 128 + kc * 256), 128, 1024),
                                  umma_desc(smem_u32(Rb + (size_t)b * TP_COLS * 128 + kc * 256), 128, 1024), idesc,
                                  (kc > 0 || a > 0) ? 1u : 0u);
            umma_commit(&mbar);
            last = t;
        }
        // the stage tile t + 1 takes held tile t - 1, whose products finished before the barrier
        if (t + 1 < nmine && tid >= TP_LOADER) load_r(t + 1, TP_LOADER, TP_THREADS - TP_LOADER);
        asm volatile("cp.async.commit_group;\n" ::);
        if (warp < 8) {
            if (t >= 1 && plive) {  // second half of tile t - 1, beside tile t's products
                const int jh = pj0 + 32 * h, nc = min(32, Sy.ncol - jh);
                float2 *p = W + (size_t)jh * m + i;
                float2 w[32];  // all 32 loads in flight at once
#pragma unroll
                for (int c = 0; c < 32; ++c) w[c] = c < nc ? p[(size_t)c * m] : make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < nc) p[(size_t)c * m] = df_sub(w[c], acc[c]);
            }
            if (t < nmine) {
                const int j0 = tile_j0(t);
                // first half of tile t: wait for its products, read the levels back, combine
                const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&mbar, t & 1, limit));
                if (!ok) {
                    s_ok = 0;
                    plive = false;
                    if (lane == 0 && atomicCAS(&st[Sy.prob].code, 0, GM_ETIMEOUT) == 0) st[Sy.prob].where = -1;
                } else {
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
                    // UPD_REST2: the diagonal tile two blocks ahead is UPD_D2's
                    const bool dt = mode == UPD_REST2 && j0 == k + nbe + 64;
                    plive = row_live && !(dt && i >= k + 2 * NBK && i < k + 3 * NBK);
                    pj0 = j0;
                    const int fe = s_fe[row], sg = t % TP_STAGES;
                    const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * h);
#pragma unroll
                    for (int c0 = 0; c0 < 32; c0 += 8) {
                        uint32_t v[S][8];
#pragma unroll
                        for (int g = 0; g < S; ++g) tmem_ld8(tb + (uint32_t)(g * TP_COLS + c0), v[g]);
                        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            // levels 3 .. S-1 in plain FP32 (their roundings stay near 2^-24
                            // of level 3, far below the digit truncation), the rest in df32
                            constexpr int G3 = S > 3 ? 3 : S - 1;
                            float lo = __uint_as_float(v[S - 1][c]) * pow2f(-7 * (S - 1));
#pragma unroll
                            for (int g = S - 2; g >= G3; --g) lo = fmaf(__uint_as_float(v[g][c]), pow2f(-7 * g), lo);
                            float2 x = make_float2(lo, 0.f);
#pragma unroll
                            for (int g = G3 - 1; g >= 0; --g)
                                x = df_add_f(x, __uint_as_float(v[g][c]) * pow2f(-7 * g));
                            acc[c0 + c] = df_scale(x, fe + s_re[sg][32 * h + c0 + c] - 12);
                        }
                    }
                }
            }
        }
    }
    // gave up: the products already issued still write tensor memory; wait (bounded) for
    // the last commit, which tracks all of them, before the memory is released
    if (tid == 256 && last >= 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        mbar_wait_bounded(&mbar, last & 1, DRAIN_POLLS);
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (warp == 8) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ----------------------------------------------------------------------------- launcher

// Launch with programmatic stream serialization when `pdl` (the kernel must call
// pdl_wait() before it reads what its predecessor in the stream writes).
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#define BLK_SPLIT_DISPATCH(split, CALL) \
    do {                                 \
        switch (split) {                 \
        case 3: { constexpr int SS = 3; CALL; } break; \
        case 4: { constexpr int SS = 4; CALL; } break; \
        case 6: { constexpr int SS = 6; CALL; } break; \
        default: { constexpr int SS = 5; CALL; } break; \
        }                                \
    } while (0)

template <int S>
static cudaError_t set_blk_attrs(int split) {
    cudaError_t e = cudaFuncSetAttribute(k_blk_factor<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)blk_factor_smem(split));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_blk_update<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)blk_update_smem(split));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_blk_update_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)blk_update_tc_smem(split));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_blk_update_tp<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)blk_update_tp_smem(split));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_blk_rfused<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)blk_rgemm_smem(split));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_blk_rfused<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)blk_rgemm_smem(split));
}

cudaError_t blk_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                         float2 *ws, int split, BlkScratch &scr, Status *st, int stage, cudaStream_t s, KTimer &kt) {
    const int nsys = (int)h_sys.size();
    cudaError_t e = cudaSuccess;
    BLK_SPLIT_DISPATCH(split, (e = set_blk_attrs<SS>(split)));
    if (e != cudaSuccess) return e;
    const size_t fsm = blk_factor_smem(split), rsm = blk_rgemm_smem(split), usm = blk_update_smem(split),
                 tsm = blk_update_tc_smem(split), psm = blk_update_tp_smem(split);
    const int nrt128 = (max_m + TC_ROWS - 1) / TC_ROWS;
    // the bulk of a block step's update (UPD_ALL, UPD_REST, UPD_REST2) on stream `on`: the
    // pipelined kernel over runs of 32-column tiles, or one CTA per 128 x 64 tile
    auto bulk_update = [&](int k, int mode, int par, cudaStream_t on) -> cudaError_t {
        const int off = mode == UPD_ALL ? 0 : 64;
        int nt = 0;
        for (const SysDesc &S : h_sys)
            if (k < S.m) nt = std::max(nt, (S.ncol - k - std::min(NBK, S.m - k) - off + TP_COLS - 1) / TP_COLS);
        if (nt <= 0) return cudaSuccess;
        if (scr.upd_tiles < 0) {
            const int ncb = (nt * TP_COLS + TC_COLS - 1) / TC_COLS;
            BLK_SPLIT_DISPATCH(split, (k_blk_update_tc<SS><<<dim3(nrt128, ncb, nsys), TILE_THREADS, tsm, on>>>(
                                          d_sys, ws, k, mode, scr.fdig[par], scr.fplane, scr.fex[par],
                                          scr.rdig[par], scr.cplane, scr.rex[par], st, scr.wait_limit)));
            return cudaGetLastError();
        }
        int tpc = scr.upd_tiles;
        if (tpc == 0) {  // one wave: a CTA per SM
            const int64_t bands = (int64_t)nsys * nrt128;
            tpc = (int)std::max<int64_t>(1, (nt * bands + scr.sms - 1) / scr.sms);
        }
        const int gy = (nt + tpc - 1) / tpc;
        BLK_SPLIT_DISPATCH(split, (k_blk_update_tp<SS><<<dim3(nrt128, gy, nsys), TP_THREADS, psm, on>>>(
                                      d_sys, ws, k, mode, tpc, scr.fdig[par], scr.fplane, scr.fex[par],
                                      scr.rdig[par], scr.cplane, scr.rex[par], st, scr.wait_limit)));
        return cudaGetLastError();
    };
    const bool la = scr.s1 && scr.s2;
    // the chain runs on s1, joined to the caller's stream on entry and exit
    cudaStream_t c = la ? scr.s1 : s;
    if (la && ((e = cudaEventRecord(scr.ev_join, s)) != cudaSuccess || (e = cudaStreamWaitEvent(c, scr.ev_join, 0))))
        return e;
    const int nrt = (max_m + 63) / 64;
    if (la && scr.early && scr.s3 && scr.x_dig2 && max_m >= 4 * NBK) {
        // Early-factor schedule.  Step k (pivot block J_k, next blocks J_k+1, J_k+2; D_j the
        // diagonal tile J_j x J_j):
        //   chain c : R of the columns J_k+1 (+ every row's F digits) -> D_k+1 -= F R on those
        //             columns (UPD_A11) -> the factor of J_k+1;
        //   s3      : R of the other columns -> D_k+2 -= F R (UPD_D2) -> the rest of column
        //             tile J_k+1 and of the row band J_k+1 (UPD_NEXT2);
        //   s2      : everything else (UPD_REST2).
        // Every tile is updated once per step.  Orderings (beyond stream order): R of step
        // k waits for UPD_NEXT2 of step k - 1 (its pivot rows and D_k's last contribution)
        // and for UPD_REST2 of step k - 2 (the digit set it overwrites, and the older
        // contributions); UPD_D2 and UPD_NEXT2 of step k wait for UPD_REST2 of step k - 1
        // (tiles it also writes); UPD_REST2 of step k waits for the R of step k.  The factor
        // of block k + 2 overwrites the first factor set after R of step k has read it (s3
        // is past that when the chain's R of step k + 1 starts).
        cudaStream_t c3 = scr.s3;
        auto fset = [&](int blk, __nv_bfloat16 *&xd, __nv_bfloat16 *&ad, int *&xe, int *&ae, float *&pm) {
            const bool two = blk & 1;
            xd = two ? scr.x_dig2 : scr.x_dig;
            ad = two ? scr.a11_dig2 : scr.a11_dig;
            xe = two ? scr.x_ex2 : scr.x_ex;
            ae = two ? scr.a11_ex2 : scr.a11_ex;
            pm = two ? scr.pmag2 : scr.pmag;
        };
        auto factor = [&](int kf, bool pdl) -> cudaError_t {
            __nv_bfloat16 *xd, *ad;
            int *xe, *ae;
            float *pm;
            fset(kf / NBK, xd, ad, xe, ae, pm);
            double fl = 0;
            for (const SysDesc &S : h_sys)
                if (kf < S.m) fl += 2.0 * std::pow((double)std::min(NBK, S.m - kf), 3.0);
            kt.begin(GM_K_PANEL, fl, c);
            cudaError_t e2 = cudaSuccess;
            BLK_SPLIT_DISPATCH(split, (e2 = launch_k(pdl, k_blk_factor<SS>, dim3(nsys), dim3(FAC_THREADS), fsm, c,
                                                     d_sys, ws, kf, xd, ad, scr.inv_plane, xe, ae, pm, st, stage)));
            kt.end(c);
            return e2;
        };
        if ((e = factor(0, false)) != cudaSuccess) return e;
        const int rb = (max_m + 127) / 128;
        for (int k = 0; k < max_m; k += NBK) {
            const int blk = k / NBK, par = blk & 1;
            __nv_bfloat16 *xd, *ad;
            int *xe, *ae;
            float *pm;
            fset(blk, xd, ad, xe, ae, pm);
            double fl_r = 0, fl_upd = 0, fl_tile = 0;
            for (const SysDesc &S : h_sys) {
                if (k >= S.m) continue;
                const double nbe = std::min(NBK, S.m - k), cols = S.ncol - k - nbe;
                fl_r += 2.0 * nbe * nbe * cols;
                fl_upd += 2.0 * nbe * ((S.m - k - nbe) * cols + (double)k * (S.ncol - S.m));
                fl_tile += 2.0 * nbe * 64.0 * 64.0;
            }
            const int cols = max_ncol - k;
            const int cb = (cols + 63) / 64;
            // ---- chain: R of the columns J_k+1 (and every row's F digits)
            if (blk > 0 && (e = cudaStreamWaitEvent(c, scr.ev_next, 0)) != cudaSuccess) return e;
            if (blk > 1 && (e = cudaStreamWaitEvent(c, scr.ev_rest2[par], 0)) != cudaSuccess) return e;
            kt.begin(GM_K_PIVROWS, fl_r * std::min(1.0, 64.0 / std::max(cols, 1)), c);
            BLK_SPLIT_DISPATCH(split, (e = launch_k(false, k_blk_rfused<SS, 2>, dim3(1 + rb, nsys), dim3(TILE_THREADS),
                                                    rsm, c, d_sys, ws, k, 1, 0, xd, ad, scr.inv_plane, xe, ae,
                                                    scr.fdig[par], scr.fplane, scr.fex[par], scr.rdig[par],
                                                    scr.cplane, scr.rex[par], pm, st)));
            if (e != cudaSuccess) return e;
            kt.end(c);
            if ((e = cudaEventRecord(scr.ev_r, c)) != cudaSuccess) return e;
            // ---- chain: the next pivot block's tile, then its factor
            kt.begin(GM_K_GJUPDATE, fl_tile, c);
            BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3(1, 1, nsys), TILE_THREADS, usm, c>>>(
                                          d_sys, ws, k, UPD_A11, nrt, scr.fdig[par], scr.fplane, scr.fex[par],
                                          scr.rdig[par], scr.cplane, scr.rex[par])));
            kt.end(c);
            if (k + NBK < max_m && (e = factor(k + NBK, !kt.timed(GM_K_GJUPDATE) && !kt.timed(GM_K_PANEL))))
                return e;
            // ---- s3: the rest of R, the diagonal tile two blocks ahead, the next band
            if ((e = cudaStreamWaitEvent(c3, scr.ev_r, 0)) != cudaSuccess) return e;
            if (cb > 1) {
                kt.begin(GM_K_PIVROWS, fl_r * std::max(0.0, 1.0 - 64.0 / std::max(cols, 1)), c3);
                if (nsys * cb <= scr.rtile32_max) {
                    const int cb32 = (cols - 64 + 31) / 32;
                    BLK_SPLIT_DISPATCH(split, (e = launch_k(false, k_blk_rfused<SS, 1>, dim3(cb32, nsys),
                                                            dim3(TILE_THREADS), rsm, c3, d_sys, ws, k, cb32, 2, xd, ad,
                                                            scr.inv_plane, xe, ae, scr.fdig[par], scr.fplane,
                                                            scr.fex[par], scr.rdig[par], scr.cplane, scr.rex[par], pm,
                                                            st)));
                } else {
                    BLK_SPLIT_DISPATCH(split, (e = launch_k(false, k_blk_rfused<SS, 2>, dim3(cb - 1, nsys),
                                                            dim3(TILE_THREADS), rsm, c3, d_sys, ws, k, cb - 1, 1, xd,
                                                            ad, scr.inv_plane, xe, ae, scr.fdig[par], scr.fplane,
                                                            scr.fex[par], scr.rdig[par], scr.cplane, scr.rex[par], pm,
                                                            st)));
                }
                if (e != cudaSuccess) return e;
                kt.end(c3);
            }
            if ((e = cudaEventRecord(scr.ev_rr, c3)) != cudaSuccess) return e;
            if (blk > 0 && (e = cudaStreamWaitEvent(c3, scr.ev_rest2[par ^ 1], 0)) != cudaSuccess) return e;
            kt.begin(GM_K_GJUPDATE, fl_tile, c3);
            BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3(1, 1, nsys), TILE_THREADS, usm, c3>>>(
                                          d_sys, ws, k, UPD_D2, nrt, scr.fdig[par], scr.fplane, scr.fex[par],
                                          scr.rdig[par], scr.cplane, scr.rex[par])));
            kt.end(c3);
            kt.begin(GM_K_GJUPDATE, std::max(0.0, fl_upd * std::min(1.0, 128.0 / std::max(cols, 1)) - 2 * fl_tile), c3);
            BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3(nrt + std::max(cb - 1, 0), 1, nsys), TILE_THREADS, usm,
                                                          c3>>>(d_sys, ws, k, UPD_NEXT2, nrt, scr.fdig[par],
                                                                scr.fplane, scr.fex[par], scr.rdig[par], scr.cplane,
                                                                scr.rex[par])));
            kt.end(c3);
            if ((e = cudaEventRecord(scr.ev_next, c3)) != cudaSuccess) return e;
            // ---- s2: the bulk of the update
            if ((e = cudaStreamWaitEvent(scr.s2, scr.ev_rr, 0)) != cudaSuccess) return e;
            if (cb > 1) {
                kt.begin(GM_K_GJUPDATE, std::max(0.0, fl_upd * std::max(0.0, 1.0 - 128.0 / std::max(cols, 1))),
                         scr.s2);
                if ((e = bulk_update(k, UPD_REST2, par, scr.s2)) != cudaSuccess) return e;
                kt.end(scr.s2);
            }
            if ((e = cudaEventRecord(scr.ev_rest2[par], scr.s2)) != cudaSuccess) return e;
        }
        // join everything into the caller's stream
        if ((e = cudaStreamWaitEvent(c, scr.ev_next, 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(c, scr.ev_rest2[0], 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(c, scr.ev_rest2[1], 0)) != cudaSuccess ||
            (e = cudaEventRecord(scr.ev_join, c)) != cudaSuccess || (e = cudaStreamWaitEvent(s, scr.ev_join, 0)))
            return e;
        return cudaGetLastError();
    }
    bool pending = false;       // the rest of the previous step's update still runs on s2
    bool next_pending = false;  // the previous step's next-block update still runs on s3
    // A11-first: the chain updates only the next pivot block's diagonal tile before that
    // block's factor; the rest of the next-block update runs on s3 beside the factor
    const bool a11 = la && scr.a11first && scr.s3;
    for (int k = 0; k < max_m; k += NBK) {
        const int par = (k / NBK) & 1;
        double fl_fac = 0, fl_r = 0, fl_upd = 0, fl_next = 0;
        for (const SysDesc &S : h_sys) {
            if (k >= S.m) continue;
            const double nbe = std::min(NBK, S.m - k), cols = S.ncol - k - nbe;
            fl_fac += 2.0 * nbe * nbe * nbe;
            fl_r += 2.0 * nbe * nbe * cols;
            // algorithmic (LU) count: the rows below the block over every remaining column,
            // the rows above it over the right-hand sides only (their matrix columns are the
            // Gauss-Jordan sweep's extra m^3/3, which an LU with back substitution avoids)
            fl_upd += 2.0 * nbe * ((S.m - k - nbe) * cols + (double)k * (S.ncol - S.m));
            const double nrow = std::max(0.0, std::min(64.0, (double)S.m - k - 64));  // next pivot rows
            fl_next += 2.0 * nbe * ((S.m - k - nbe) * std::min(64.0, cols) + nrow * std::max(0.0, cols - 64));
        }
        const int cols = max_ncol - k;
        const int cb = (cols + 63) / 64, rb = (max_m + 127) / 128;
        kt.begin(GM_K_PANEL, fl_fac, c);
        // programmatic launches where the predecessor in the stream is the kernel waited on
        // (not with timing events between launches, not after the entry join)
        const bool pdl = k > 0 && !kt.timed(GM_K_GJUPDATE) && !kt.timed(GM_K_PANEL);
        BLK_SPLIT_DISPATCH(split, (e = launch_k(pdl, k_blk_factor<SS>, dim3(nsys), dim3(FAC_THREADS), fsm, c, d_sys,
                                                ws, k, scr.x_dig, scr.a11_dig, scr.inv_plane, scr.x_ex, scr.a11_ex,
                                                scr.pmag, st, stage)));
        if (e != cudaSuccess) return e;
        kt.end(c);
        // R writes digit set `par`, which the rest of the update two steps back read: that
        // finished before the previous step's next-block update (below) started
        bool pdl_r = !kt.timed(GM_K_PANEL) && !kt.timed(GM_K_PIVROWS);
        if (next_pending) {  // R reads the pivot rows and the F column the s3 update writes
            if ((e = cudaStreamWaitEvent(c, scr.ev_next, 0)) != cudaSuccess) return e;
            next_pending = false;
            pdl_r = false;
        }
        kt.begin(GM_K_PIVROWS, fl_r, c);
        // 32-column R tiles while the step would leave most SMs idle
        if (nsys * cb <= scr.rtile32_max) {
            const int cb32 = (cols + 31) / 32;
            BLK_SPLIT_DISPATCH(split, (e = launch_k(pdl_r, k_blk_rfused<SS, 1>, dim3(cb32 + rb, nsys),
                                                    dim3(TILE_THREADS), rsm, c, d_sys, ws, k, cb32, 0, scr.x_dig,
                                                    scr.a11_dig, scr.inv_plane, scr.x_ex, scr.a11_ex, scr.fdig[par],
                                                    scr.fplane, scr.fex[par], scr.rdig[par], scr.cplane,
                                                    scr.rex[par], scr.pmag, st)));
        } else {
            BLK_SPLIT_DISPATCH(split, (e = launch_k(pdl_r, k_blk_rfused<SS, 2>, dim3(cb + rb, nsys),
                                                    dim3(TILE_THREADS), rsm, c, d_sys, ws, k, cb, 0, scr.x_dig,
                                                    scr.a11_dig, scr.inv_plane, scr.x_ex, scr.a11_ex, scr.fdig[par],
                                                    scr.fplane, scr.fex[par], scr.rdig[par], scr.cplane,
                                                    scr.rex[par], scr.pmag, st)));
        }
        if (e != cudaSuccess) return e;
        kt.end(c);
        const dim3 gu(nrt, cb, nsys);
        if (la && cb >= 2 && (e = cudaEventRecord(scr.ev_r, c)) != cudaSuccess) return e;
        // this step's update rewrites tiles the rest of the previous step's update touches
        if (pending) {
            if ((e = cudaStreamWaitEvent(c, scr.ev_rest, 0)) != cudaSuccess) return e;
            if (a11 && cb >= 2 && (e = cudaStreamWaitEvent(scr.s3, scr.ev_rest, 0)) != cudaSuccess) return e;
            pending = false;
        }
        if (!la || cb < 2) {
            kt.begin(GM_K_GJUPDATE, fl_upd, c);
            if ((e = bulk_update(k, UPD_ALL, par, c)) != cudaSuccess) return e;
            kt.end(c);
            continue;
        }
        // look-ahead: everything the next factor and R kernel read (the next block's
        // columns and its pivot rows) on s1, the rest on s2, overlapping the next factor and
        // R kernel (disjoint tiles, the other digit set)
        if (a11) {
            // chain: the next pivot block's diagonal tile only, so that its factor starts
            // at once; s3: the rest of its column and of its row band (read by the next R
            // kernel, which waits for it)
            double fl_t = 0;
            for (const SysDesc &S : h_sys)
                if (k + NBK < S.m) fl_t += 2.0 * std::min(NBK, S.m - k) * 64.0 * std::min(64, S.m - k - NBK);
            kt.begin(GM_K_GJUPDATE, fl_t, c);
            BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3(1, 1, nsys), TILE_THREADS, usm, c>>>(
                                          d_sys, ws, k, UPD_A11, nrt, scr.fdig[par], scr.fplane, scr.fex[par],
                                          scr.rdig[par], scr.cplane, scr.rex[par])));
            kt.end(c);
            if ((e = cudaStreamWaitEvent(scr.s3, scr.ev_r, 0)) != cudaSuccess) return e;
            kt.begin(GM_K_GJUPDATE, std::max(0.0, fl_next - fl_t), scr.s3);
            BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3(nrt + cb - 1, 1, nsys), TILE_THREADS, usm, scr.s3>>>(
                                          d_sys, ws, k, UPD_NEXT2, nrt, scr.fdig[par], scr.fplane, scr.fex[par],
                                          scr.rdig[par], scr.cplane, scr.rex[par])));
            kt.end(scr.s3);
            if ((e = cudaEventRecord(scr.ev_next, scr.s3)) != cudaSuccess) return e;
            next_pending = true;
        } else {
            kt.begin(GM_K_GJUPDATE, fl_next, c);
            BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3(nrt + cb - 1, 1, nsys), TILE_THREADS, usm, c>>>(
                                          d_sys, ws, k, UPD_NEXT, nrt, scr.fdig[par], scr.fplane, scr.fex[par],
                                          scr.rdig[par], scr.cplane, scr.rex[par])));
            kt.end(c);
        }
        if ((e = cudaStreamWaitEvent(scr.s2, scr.ev_r, 0)) != cudaSuccess) return e;
        kt.begin(GM_K_GJUPDATE, fl_upd - fl_next, scr.s2);
        if ((e = bulk_update(k, UPD_REST, par, scr.s2)) != cudaSuccess) return e;
        kt.end(scr.s2);
        if ((e = cudaEventRecord(scr.ev_rest, scr.s2)) != cudaSuccess) return e;
        pending = true;
    }
    if (pending && (e = cudaStreamWaitEvent(c, scr.ev_rest, 0)) != cudaSuccess) return e;
    if (next_pending && (e = cudaStreamWaitEvent(c, scr.ev_next, 0)) != cudaSuccess) return e;
    if (la && ((e = cudaEventRecord(scr.ev_join, c)) != cudaSuccess || (e = cudaStreamWaitEvent(s, scr.ev_join, 0))))
        return e;
    return cudaGetLastError();
}

}  // namespace gm
