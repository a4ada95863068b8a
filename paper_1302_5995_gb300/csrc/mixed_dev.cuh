// Device helpers of the mixed-precision kernels: double-float (df32) arithmetic, the
// signed 7-bit digit split, mma.sync digit products, and digit-plane GEMM tiles.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gm_internal.h"

namespace gm {

// ----------------------------------------------------------------------------- df32

__device__ __forceinline__ float2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    float2 t = two_sum(a.y, b.y);
    s.y = __fadd_rn(s.y, t.x);
    s = fast_two_sum(s.x, s.y);
    s.y = __fadd_rn(s.y, t.y);
    return fast_two_sum(s.x, s.y);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ float2 df_add_f(float2 a, float b) {
    float2 s = two_sum(a.x, b);
    s.y = __fadd_rn(s.y, a.y);
    return fast_two_sum(s.x, s.y);
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
    float q = __fdiv_rn(a.x, b.x);
    float2 r = df_sub(a, df_mul(make_float2(q, 0.f), b));
    float q2 = __fdiv_rn(r.x, b.x);
    return fast_two_sum(q, q2);
}
__device__ __forceinline__ float2 df_from_d(double x) {
    float hi = __double2float_rn(x);
    float lo = __double2float_rn(x - (double)hi);
    return make_float2(hi, lo);
}
__device__ __forceinline__ double df_to_d(float2 a) { return (double)a.x + (double)a.y; }
// 2^p as a float for -126 <= p <= 127 (built from its exponent bits), and x 2^p for
// -252 <= p <= 254 by two such factors: exact while the result stays a normal float
// (the only case here), at two multiplications instead of a library scaling call
__device__ __forceinline__ float pow2f(int p) { return __int_as_float((p + 127) << 23); }
__device__ __forceinline__ float2 df_scale(float2 a, int p) {
    const float f1 = pow2f(p >> 1), f2 = pow2f(p - (p >> 1));
    return make_float2(a.x * f1 * f2, a.y * f1 * f2);
}

// ----------------------------------------------------------------------------- tcgen05

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle, version 1 (start, LBO and SBO in
// 16-byte units; LBO = distance of core matrices along k, SBO = along the rows).
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B (both K-major).
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) += / = A B^T for one 16-k step (acc = 0 starts the accumulator).
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(void *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(mbar)));
}

// Default poll count of the bounded waits, and the fixed bound of the waits a kernel
// makes, after giving up, for its own copies and products still in flight.
constexpr int WAIT_POLLS = 1 << 22;
constexpr int DRAIN_POLLS = 1 << 24;

// Wait for completion `parity` of an mbarrier, giving up after `limit` polls (false).
__device__ __forceinline__ bool mbar_wait_bounded(void *mbar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(mbar)), "r"(parity));
    return done != 0;
}

// Eight fp32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t v[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start while its predecessor in the stream finishes; pdl_wait() blocks until the
// predecessor has completed and its writes are visible (a no-op without the attribute),
// pdl_trigger() lets this kernel's own dependent start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ----------------------------------------------------------------------------- digits

// Exponent e with |x| < 2^e for every x of a set whose largest |hi| is m (0 -> 0).
__device__ __forceinline__ int exp_of_max(float m) {
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    return e;
}

// S signed digits of x 2^(6-e): d_0 + 2^-7 d_1 + ..., |d_s| <= 64.
template <int S>
__device__ __forceinline__ void digits(float2 x, int e, float d[S]) {
    const float2 t = df_scale(x, 6 - e);
    float th = t.x, tl = t.y;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float q = rintf(th);
        d[s] = q;
        float2 r = two_sum(__fsub_rn(th, q), tl);
        th = __fmul_rn(r.x, 128.f);
        tl = __fmul_rn(r.y, 128.f);
    }
}

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared-memory digit tiles: A as [S][BM][KP] (k fastest), B as [S][BN][KP]; KP = 24
// bf16 (16 used) makes the fragment loads bank-conflict free.
constexpr int KP = 24;

// One warp accumulates a 32 x (8 NT) block: 2 m16 tiles x NT n8 tiles, S levels.  Tiles
// are [S][rows][LD] (k fastest); the 16 k of this step start at As / Bs.
template <int S, int LD = KP, int NT = 4>
__device__ __forceinline__ void warp_mma_levels(const __nv_bfloat16 *As, const __nv_bfloat16 *Bs, int BM, int BN,
                                                int wm, int wn, float acc[S][2][NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const __nv_bfloat16 *p = As + ((size_t)s * BM + wm + mt * 16 + g) * LD + 2 * t;
            a[mt][0] = *(const uint32_t *)(p);
            a[mt][1] = *(const uint32_t *)(p + 8 * LD);
            a[mt][2] = *(const uint32_t *)(p + 8);
            a[mt][3] = *(const uint32_t *)(p + 8 * LD + 8);
        }
#pragma unroll
        for (int u = 0; u < S; ++u) {
            if (s + u >= S) continue;
            uint32_t b[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const __nv_bfloat16 *p = Bs + ((size_t)u * BN + wn + nt * 8 + g) * LD + 2 * t;
                b[nt][0] = *(const uint32_t *)(p);
                b[nt][1] = *(const uint32_t *)(p + 8);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
                    mma_bf16(acc[s + u][mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
        }
    }
}

// df32 value of one output position from its S exact level sums and the scale.
template <int S, int NT = 4>
__device__ __forceinline__ float2 combine_levels(const float acc[S][2][NT][4], int mt, int nt, int c, int p) {
    float2 v = make_float2(acc[S - 1][mt][nt][c] * pow2f(-7 * (S - 1)), 0.f);
#pragma unroll
    for (int g = S - 2; g >= 0; --g) v = df_add_f(v, acc[g][mt][nt][c] * pow2f(-7 * g));
    return df_scale(v, p);
}

// Position within the warp block of accumulator element (mt, nt, c).
__device__ __forceinline__ void acc_pos(int mt, int nt, int c, int &r, int &col) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    r = mt * 16 + g + (c >= 2 ? 8 : 0);
    col = nt * 8 + 2 * t + (c & 1);
}

// ----------------------------------------------------------------------------- stencil

__device__ __forceinline__ double stencil_w_mx(const double *__restrict__ b, const double *__restrict__ c,
                                               const double *__restrict__ d, double ih, int g, int dir) {
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

__device__ __forceinline__ void record_pivot_mx(Status *st, double piv, int stage) {
    double ap = fabs(piv);
    if (!(ap > 0.0) || !isfinite(ap)) {
        if (atomicCAS(&st->code, 0, GM_ESINGULAR) == 0) st->where = stage;
        return;
    }
    atomicMin(&st->min_piv, (unsigned long long)__double_as_longlong(ap));
}

struct MergeTabMx {
    const int *p3, *p4, *g3, *g4, *p1, *q1, *p2, *q2, *x12;
};
__device__ __forceinline__ MergeTabMx merge_tab_mx(const MergeDesc &M, const int *tab) {
    const int *t = tab + M.tab;
    MergeTabMx T;
    T.p3 = t; T.p4 = t + M.sp; T.g3 = t + 2 * M.sp; T.g4 = t + 3 * M.sp;
    T.p1 = t + 4 * M.sp; T.q1 = T.p1 + M.n1; T.p2 = T.q1 + M.n1; T.q2 = T.p2 + M.n2;
    T.x12 = T.q2 + M.n2;
    return T;
}

// ----------------------------------------------------------------------------- digit planes

// A digit matrix holds, for each of S digits, a plane of rows x kpad bf16 values
// (k fastest, zero beyond K), plus one exponent per row: element (s, row, k) is at
// dig[s * plane + row * kpad + k].  kpad is a multiple of 16.

// One lane-strided warp slices a row of K df32 values, produced by `get(k)`.
// Element (row, k) of a digit plane stored by 128-row x 16-k tiles, each tile in the
// tensor cores' K-major core-matrix order (8 x 8 blocks of 128 bytes, k-block fastest
// within a row group): a tile is one contiguous 4 KB bulk copy.
__device__ __forceinline__ int64_t tiled_idx(int row, int k, int kpad) {
    return ((int64_t)(row >> 7) * (kpad >> 4) + (k >> 4)) * 2048 + ((row & 127) >> 3) * 128 + ((k & 15) >> 3) * 64 +
           (row & 7) * 8 + (k & 7);
}

template <int S, class Get>
__device__ __forceinline__ void warp_slice_row(Get get, int K, int kpad, __nv_bfloat16 *dig, int64_t plane, int64_t row,
                                               int *ex, bool tiled = false) {
    const int lane = threadIdx.x & 31;
    float mx = 0.f;
    for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(get(k).x));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = exp_of_max(mx * 1.0000001f);
    if (lane == 0) ex[row] = e;
    for (int k = lane; k < kpad; k += 32) {
        float d[S];
        float2 v = k < K ? get(k) : make_float2(0.f, 0.f);
        digits<S>(v, e, d);
        const int64_t at = tiled ? tiled_idx((int)row, k, kpad) : row * kpad + k;
#pragma unroll
        for (int s = 0; s < S; ++s) dig[(int64_t)s * plane + at] = __float2bfloat16_rn(d[s]);
    }
}

// 64 rows x 16 k of every digit plane into shared memory ([S][64][KP]); 128 threads.
template <int S>
__device__ __forceinline__ void load_digit_tile(const __nv_bfloat16 *__restrict__ dig, int64_t plane, int kpad,
                                                int r0, int nrows, int k0, __nv_bfloat16 *sm) {
    const int row = threadIdx.x >> 1, half = threadIdx.x & 1;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < nrows) v = *(const uint4 *)(dig + (int64_t)s * plane + (int64_t)(r0 + row) * kpad + k0 + half * 8);
        *(uint4 *)(sm + ((size_t)s * 64 + row) * KP + half * 8) = v;
    }
}

// C(i, j) = sum_k A(i, k) B(k, j) for a 64 x 64 tile from two digit matrices (A by rows,
// B by columns), K in chunks of at most 512 (exact level sums).  After each chunk the
// df32 partial results are handed to epi(r[4], c[4], value[4], first) four at a time (one
// m16 x n8 fragment: r, c the positions in the tile, see acc_pos), first = this is the
// first chunk; the caller accumulates (so no second register tile is live beside the
// level sums) and can issue a group's memory reads together.
// Warp w owns rows (w & 1) * 32 and columns (w >> 1) * 32.
template <int S, class Epi>
__device__ __forceinline__ void digit_gemm_chunks(const __nv_bfloat16 *__restrict__ Ad, int64_t aplane, int akpad,
                                                  int i0, int M, const int *__restrict__ aex,
                                                  const __nv_bfloat16 *__restrict__ Bd, int64_t bplane, int bkpad,
                                                  int j0, int N, const int *__restrict__ bex, int K,
                                                  __nv_bfloat16 *As, __nv_bfloat16 *Bs, Epi &&epi) {
    const int warp = threadIdx.x >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
    const int mrows = min(64, M - i0), ncols = min(64, N - j0);
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += 512) {
        const int kend = min(K, k0 + 512);
        float acc[S][2][4][4];
#pragma unroll
        for (int g = 0; g < S; ++g)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[g][mt][nt][c] = 0.f;
#pragma unroll 1
        for (int t0 = k0; t0 < kend; t0 += 16) {
            __syncthreads();
            load_digit_tile<S>(Ad, aplane, akpad, i0, mrows, t0, As);
            load_digit_tile<S>(Bd, bplane, bkpad, j0, ncols, t0, Bs);
            __syncthreads();
            warp_mma_levels<S>(As, Bs, 64, 64, wm, wn, acc);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                int rr[4], cc[4];
                float2 vv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    int r, cl;
                    acc_pos(mt, nt, c, r, cl);
                    const int i = min(i0 + wm + r, M - 1), j = min(j0 + wn + cl, N - 1);
                    rr[c] = wm + r;
                    cc[c] = wn + cl;
                    vv[c] = combine_levels<S>(acc, mt, nt, c, aex[i] + bex[j] - 12);
                }
                epi(rr, cc, vv, k0 == 0);
            }
    }
}

// Pipelined variant of digit_gemm_chunks for 256 threads (a 2 x 4 warp grid, 32 x 16 per
// warp): K-tiles of 32 move by cp.async through a three-stage ring in dynamic shared
// memory, so the copy of tile t + 2 overlaps the products of tile t (one barrier per
// tile).  Same K chunks of at most 512 and the same epilogue interface.
constexpr int PIPE_K = 32, PIPE_KP = 40, PIPE_STAGES = 3, PIPE_THREADS = 256, PIPE_NT = 2;
// (40 bf16 = 20 words per row: the fragment loads of eight rows x four words hit 32 banks)
__host__ __device__ constexpr size_t pipe_smem_bytes(int S) {
    return (size_t)PIPE_STAGES * 2 * S * 64 * PIPE_KP * sizeof(__nv_bfloat16);
}

// Rows r0 .. r0 + 63 (zero beyond nrows or kpad) of columns t0 .. t0 + 31 of every digit plane.
template <int S>
__device__ __forceinline__ void pipe_load(const __nv_bfloat16 *__restrict__ dig, int64_t plane, int kpad, int r0,
                                          int nrows, int t0, __nv_bfloat16 *sm) {
    for (int e = threadIdx.x; e < S * 64 * 4; e += PIPE_THREADS) {
        const int q = e & 3, row = (e >> 2) & 63, s = e >> 8;
        const int kk = t0 + q * 8;
        const bool ok = row < nrows && kk < kpad;
        const __nv_bfloat16 *src = dig + (int64_t)s * plane + (int64_t)(r0 + (ok ? row : 0)) * kpad + (ok ? kk : 0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(sm + ((size_t)s * 64 + row) * PIPE_KP + q * 8);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0));
    }
}

template <int S, class Epi>
__device__ __forceinline__ void digit_gemm_pipe(const __nv_bfloat16 *__restrict__ Ad, int64_t aplane, int akpad,
                                                int i0, int M, const int *__restrict__ aex,
                                                const __nv_bfloat16 *__restrict__ Bd, int64_t bplane, int bkpad,
                                                int j0, int N, const int *__restrict__ bex, int K,
                                                __nv_bfloat16 *smem, Epi &&epi) {
    const int warp = threadIdx.x >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 8 * PIPE_NT;
    const int mrows = min(64, M - i0), ncols = min(64, N - j0);
    const int ntiles = (K + PIPE_K - 1) / PIPE_K;
    constexpr size_t PLANES = (size_t)S * 64 * PIPE_KP;
    auto load = [&](int t) {
        __nv_bfloat16 *st = smem + (size_t)(t % PIPE_STAGES) * 2 * PLANES;
        pipe_load<S>(Ad, aplane, akpad, i0, mrows, t * PIPE_K, st);
        pipe_load<S>(Bd, bplane, bkpad, j0, ncols, t * PIPE_K, st + PLANES);
    };
#pragma unroll
    for (int t = 0; t < PIPE_STAGES - 1; ++t) {
        if (t < ntiles) load(t);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    float acc[S][2][PIPE_NT][4];
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < PIPE_NT; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[g][mt][nt][c] = 0.f;
#pragma unroll 1
    for (int t = 0; t < ntiles; ++t) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(PIPE_STAGES - 2));  // tile t has landed
        __syncthreads();  // ... for every thread, and tile t - 1's products are done
        if (t + PIPE_STAGES - 1 < ntiles) load(t + PIPE_STAGES - 1);
        asm volatile("cp.async.commit_group;\n" ::);
        const __nv_bfloat16 *As = smem + (size_t)(t % PIPE_STAGES) * 2 * PLANES, *Bs = As + PLANES;
        warp_mma_levels<S, PIPE_KP, PIPE_NT>(As, Bs, 64, 64, wm, wn, acc);
        if (t * PIPE_K + 16 < K) warp_mma_levels<S, PIPE_KP, PIPE_NT>(As + 16, Bs + 16, 64, 64, wm, wn, acc);
        const int tend = (t + 1) * PIPE_K;
        if (tend % 512 == 0 || t == ntiles - 1) {  // end of a K chunk: hand the results over
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < PIPE_NT; ++nt) {
                    int rr[4], cc[4];
                    float2 vv[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        int r, cl;
                        acc_pos(mt, nt, c, r, cl);
                        const int i = min(i0 + wm + r, M - 1), j = min(j0 + wn + cl, N - 1);
                        rr[c] = wm + r;
                        cc[c] = wn + cl;
                        vv[c] = combine_levels<S, PIPE_NT>(acc, mt, nt, c, aex[i] + bex[j] - 12);
                        acc[0][mt][nt][c] = 0.f;
                    }
#pragma unroll
                    for (int g = 1; g < S; ++g)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[g][mt][nt][c] = 0.f;
                    epi(rr, cc, vv, tend <= 512);
                }
        }
    }
}

}  // namespace gm
