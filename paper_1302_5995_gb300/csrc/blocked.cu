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

constexpr int FAC_THREADS = 1024;

template <int S>
__global__ void __launch_bounds__(FAC_THREADS)
k_blk_factor(const SysDesc *__restrict__ sys, const float2 *__restrict__ ws, int k, __nv_bfloat16 *__restrict__ x_dig,
             __nv_bfloat16 *__restrict__ a_dig, int64_t plane, int *__restrict__ x_ex, int *__restrict__ a_ex,
             float *__restrict__ pmag, Status *st, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Aug = (float *)smem_raw;                 // [64][129] FP32 [A11 | I]
    float2 *Adf = (float2 *)(Aug + 64 * 129 + 64);  // [64][LDF] A11 (df32)
    __shared__ float fcol[64];
    __shared__ int s_p;
    const SysDesc Sy = sys[blockIdx.x];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    const float2 *W = ws + Sy.off;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5;
    for (int e = tid; e < 64 * 64; e += nt) {  // A11, padded with the identity beyond nbe
        const int i = e % 64, j = e / 64;
        float2 v = (i < nbe && j < nbe) ? W[(size_t)(k + j) * m + k + i] : make_float2(i == j ? 1.f : 0.f, 0.f);
        Adf[i * LDF + j] = v;
        Aug[i * 129 + j] = v.x;
        Aug[i * 129 + 64 + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    // Gauss-Jordan on [A11 | I] with partial pivoting among the unused rows; rows are
    // not moved: pivot row of column t is prow_of[t], and X0 row t is that row's right half.
    __shared__ int prow_of[64];
    __shared__ unsigned long long used;
    __shared__ float prow[128];
    if (tid == 0) used = 0ull;
    __syncthreads();
    for (int t = 0; t < 64; ++t) {
        if (warp == 0) {
            float best = -1.f;
            int bi = 64;
            for (int r = tid; r < 64; r += 32) {
                if ((used >> r) & 1ull) continue;
                float v = fabsf(Aug[r * 129 + t]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                float v2 = __shfl_down_sync(0xffffffffu, best, o);
                int i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
            }
            if (tid == 0) {
                if (bi >= 64) {  // no candidate (cannot happen: 64 - t unused rows remain)
                    for (bi = 0; bi < 64 && ((used >> bi) & 1ull); ++bi) {}
                    if (bi >= 64) bi = 0;
                }
                s_p = bi;
                prow_of[t] = bi;
                used |= 1ull << bi;
                if (t < nbe) pmag[(size_t)blockIdx.x * 64 + t] = best;
            }
        }
        __syncthreads();
        const int p = s_p;
        const float pv = Aug[p * 129 + t];
        const float ipv = pv != 0.f ? 1.f / pv : 0.f;
        if (tid < 128) prow[tid] = Aug[p * 129 + tid] * ipv;
        else if (tid < 192) fcol[tid - 128] = Aug[(tid - 128) * 129 + t];
        __syncthreads();
        {  // thread owns column c, rows r = g, g + G, ...; eliminated columns (c <= t) stay
            const int c = tid & 127, G = nt >> 7;
            if (c > t || c >= 64) {
                const float pc = prow[c];
                for (int r = tid >> 7; r < 64; r += G)
                    Aug[r * 129 + c] = (r == p) ? pc : Aug[r * 129 + c] - fcol[r] * pc;
            } else if (c == t) {
                for (int r = tid >> 7; r < 64; r += G) Aug[r * 129 + c] = (r == p) ? 1.f : 0.f;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        float mn = 3.0e38f;
        for (int t = 0; t < nbe; ++t) mn = fminf(mn, pmag[(size_t)blockIdx.x * 64 + t]);
        record_pivot_mx(st + Sy.prob, (double)mn, stage);
    }
    // digit planes of the rows of X0 and of A11 (K = 64), one warp per row
    for (int i = warp; i < 128; i += nt / 32) {
        if (i < 64) {
            const int64_t row = (int64_t)blockIdx.x * 64 + i;
            const int src = prow_of[i];
            warp_slice_row<S>([&](int q) { return make_float2(Aug[src * 129 + 64 + q], 0.f); }, 64, 64, x_dig,
                              plane, row, x_ex);
        } else {
            const int ii = i - 64;
            const int64_t row = (int64_t)blockIdx.x * 64 + ii;
            warp_slice_row<S>([&](int q) { return Adf[ii * LDF + q]; }, 64, 64, a_dig, plane, row, a_ex);
        }
    }
}

size_t blk_factor_smem(int split) {
    (void)split;
    return (size_t)(64 * 129 + 64) * sizeof(float) + 64 * LDF * sizeof(float2);
}

// ----------------------------------------------------------------------------- R = A11^{-1} A12

// Column exponents of a 64 x 64 df32 shared tile D[t][jj] (rows t >= nrow count as 0).
__device__ __forceinline__ void col_exps64(const float2 *D, int *ex) {
    if (threadIdx.x < 64) {
        float mx = 0.f;
        for (int t = 0; t < NBK; ++t) mx = fmaxf(mx, fabsf(D[t * LDF + threadIdx.x].x));
        ex[threadIdx.x] = exp_of_max(mx * 1.0000001f);
    }
}

// P = A D for a 64 x 64 x 64 product: A by rows from global digit planes (64 rows at
// adig, exponents aex), D a df32 shared tile sliced by columns on the fly (exponents exB).
template <int S>
__device__ __forceinline__ void gemm64_gd(const __nv_bfloat16 *__restrict__ adig, int64_t plane,
                                          const int *__restrict__ aex, const float2 *D, const int *exB,
                                          __nv_bfloat16 *As, __nv_bfloat16 *Bs, float2 res[2][4][4]) {
    const int tid = threadIdx.x, warp = tid >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
    float acc[S][2][4][4];
#pragma unroll
    for (int g = 0; g < S; ++g)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[g][mt][nt][c] = 0.f;
    for (int t0 = 0; t0 < NBK; t0 += 16) {
        __syncthreads();
        load_digit_tile<S>(adig, plane, NBK, 0, 64, t0, As);
        for (int e = tid; e < 64 * 16; e += 128) {
            const int jj = e >> 4, t = e & 15;
            float d[S];
            digits<S>(D[(t0 + t) * LDF + jj], exB[jj], d);
#pragma unroll
            for (int s = 0; s < S; ++s) Bs[((size_t)s * 64 + jj) * KP + t] = __float2bfloat16_rn(d[s]);
        }
        __syncthreads();
        warp_mma_levels<S>(As, Bs, 64, 64, wm, wn, acc);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                res[mt][nt][c] = combine_levels<S>(acc, mt, nt, c, aex[wm + r] + exB[wn + cl] - 12);
            }
}

// Blocks [0, cb): 64 columns right of the pivot block each:
//   R0 = X0 A12,  E = A12 - A11 R0,  R = R0 + X0 E  (one refinement step),
// R written into the pivot rows and cut into column digit planes for the update.
// Blocks [cb, cb + rb): 128 rows each: F = W(i, J) (zero inside J) into row digit planes,
// with the growth check against the block pivots.
template <int S>
__global__ void __launch_bounds__(128)
k_blk_rfused(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, int cb,
             const __nv_bfloat16 *__restrict__ x_dig, const __nv_bfloat16 *__restrict__ a11_dig, int64_t plane,
             const int *__restrict__ x_ex, const int *__restrict__ a11_ex, __nv_bfloat16 *__restrict__ fdig,
             int64_t fplane, int *__restrict__ fex, __nv_bfloat16 *__restrict__ rdig, int64_t cplane,
             int *__restrict__ rex, const float *__restrict__ pmag, Status *__restrict__ st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SysDesc Sy = sys[blockIdx.y];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    float2 *W = ws + Sy.off;
    if ((int)blockIdx.x >= cb) {
        const int i = ((int)blockIdx.x - cb) * 128 + threadIdx.x;
        if (i >= m) return;
        const bool inJ = i >= k && i < k + nbe;
        float mx = 0.f;
        bool grow = false;
        for (int t = 0; t < nbe; ++t) {
            const float v = inJ ? 0.f : fabsf(W[(size_t)(k + t) * m + i].x);
            mx = fmaxf(mx, v);
            if (i >= k + nbe && v > 16.f * pmag[(size_t)blockIdx.y * 64 + t]) grow = true;
        }
        if (grow) atomicOr(&st[Sy.prob].growth, 1);
        const int e = exp_of_max(mx * 1.0000001f);
        const int64_t row = Sy.roff + i;
        fex[row] = e;
        for (int t = 0; t < NBK; ++t) {
            float d[S];
            digits<S>((inJ || t >= nbe) ? make_float2(0.f, 0.f) : W[(size_t)(k + t) * m + i], e, d);
#pragma unroll
            for (int s = 0; s < S; ++s) fdig[(int64_t)s * fplane + row * NBK + t] = __float2bfloat16_rn(d[s]);
        }
        return;
    }
    const int j0 = k + nbe + blockIdx.x * 64;
    if (j0 >= Sy.ncol) return;
    __nv_bfloat16 *As = (__nv_bfloat16 *)smem_raw;
    __nv_bfloat16 *Bs = As + S * 64 * KP;
    float2 *Ad = (float2 *)(Bs + S * 64 * KP);  // [64][LDF]: A12, then E
    float2 *Rd = Ad + 64 * LDF;                  // [64][LDF]: R0, then R
    __shared__ int exB[64];
    const int tid = threadIdx.x, warp = tid >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
    for (int e = tid; e < 64 * 64; e += 128) {
        const int t = e & 63, jj = e >> 6, j = j0 + jj;
        Ad[t * LDF + jj] = (t < nbe && j < Sy.ncol) ? W[(size_t)j * m + k + t] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    col_exps64(Ad, exB);
    const __nv_bfloat16 *xd = x_dig + (int64_t)blockIdx.y * 64 * NBK, *ad = a11_dig + (int64_t)blockIdx.y * 64 * NBK;
    const int *xe = x_ex + blockIdx.y * 64, *ae = a11_ex + blockIdx.y * 64;
    float2 res[2][4][4];
    gemm64_gd<S>(xd, plane, xe, Ad, exB, As, Bs, res);  // R0 = X0 A12
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                Rd[(wm + r) * LDF + wn + cl] = (wm + r < nbe) ? res[mt][nt][c] : make_float2(0.f, 0.f);
            }
    __syncthreads();
    col_exps64(Rd, exB);
    gemm64_gd<S>(ad, plane, ae, Rd, exB, As, Bs, res);  // A11 R0
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                float2 *p = Ad + (wm + r) * LDF + wn + cl;
                *p = (wm + r < nbe) ? df_sub(*p, res[mt][nt][c]) : make_float2(0.f, 0.f);  // E
            }
    __syncthreads();
    col_exps64(Ad, exB);
    __shared__ int cmax[64], rmax[64];  // column maxima of |X0 E| and |R| (float bits, >= 0)
    if (tid < 64) cmax[tid] = rmax[tid] = 0;
    gemm64_gd<S>(xd, plane, xe, Ad, exB, As, Bs, res);  // X0 E
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                const int t = wm + r, jj = wn + cl, j = j0 + jj;
                float2 v = (t < nbe) ? df_add(Rd[t * LDF + jj], res[mt][nt][c]) : make_float2(0.f, 0.f);
                Rd[t * LDF + jj] = v;
                if (t < nbe && j < Sy.ncol) {
                    W[(size_t)j * m + k + t] = v;
                    atomicMax(&cmax[jj], __float_as_int(fabsf(res[mt][nt][c].x)));
                    atomicMax(&rmax[jj], __float_as_int(fabsf(v.x)));
                }
            }
    __syncthreads();
    // The refinement step leaves an error of about rho^2 |R|, where rho = |X0 E| / |R|
    // is its contraction factor (kappa(A11) times the FP32 accuracy of X0).  A column
    // with rho above 2^-16 would keep more than about 2^-32 |R|: raise the flag that sends
    // the build to partial pivoting.
    if (tid < 64 && __int_as_float(cmax[tid]) > 0x1p-16f * __int_as_float(rmax[tid])) atomicOr(&st[Sy.prob].growth, 1);
    col_exps64(Rd, exB);
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += 128) {  // column digit planes of R
        const int jj = e >> 6, t = e & 63, j = j0 + jj;
        if (j >= Sy.ncol) continue;
        const int64_t row = Sy.coff + j;
        if (t == 0) rex[row] = exB[jj];
        float d[S];
        digits<S>(Rd[t * LDF + jj], exB[jj], d);
#pragma unroll
        for (int s = 0; s < S; ++s) rdig[(int64_t)s * cplane + row * NBK + t] = __float2bfloat16_rn(d[s]);
    }
}

size_t blk_rgemm_smem(int split) { return 2 * (size_t)split * 64 * KP * 2 + 2 * 64 * LDF * sizeof(float2); }

// ----------------------------------------------------------------------------- update

template <int S>
__global__ void __launch_bounds__(128)
k_blk_update(const SysDesc *__restrict__ sys, float2 *__restrict__ ws, int k, const __nv_bfloat16 *__restrict__ fdig,
             int64_t fplane, const int *__restrict__ fex, const __nv_bfloat16 *__restrict__ rdig, int64_t rplane,
             const int *__restrict__ rex) {
    __shared__ __align__(16) __nv_bfloat16 As[S * 64 * KP];
    __shared__ __align__(16) __nv_bfloat16 Bs[S * 64 * KP];
    const SysDesc Sy = sys[blockIdx.z];
    const int m = Sy.m;
    if (k >= m) return;
    const int nbe = min(NBK, m - k);
    const int i0 = blockIdx.x * 64, j0 = k + nbe + blockIdx.y * 64;
    if (i0 >= m || j0 >= Sy.ncol) return;
    float2 *W = ws + Sy.off;
    float2 res[2][4][4];
    digit_gemm_tile<S>(fdig + (int64_t)Sy.roff * NBK, fplane, NBK, i0, m, fex + Sy.roff, rdig + (int64_t)Sy.coff * NBK,
                       rplane, NBK, j0, Sy.ncol, rex + Sy.coff, NBK, As, Bs, res);
    const int warp = threadIdx.x >> 5, wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int r, cl;
                acc_pos(mt, nt, c, r, cl);
                const int i = i0 + wm + r, j = j0 + wn + cl;
                if (i >= m || j >= Sy.ncol || (i >= k && i < k + nbe)) continue;
                float2 *p = W + (size_t)j * m + i;
                *p = df_sub(*p, res[mt][nt][c]);
            }
}

// ----------------------------------------------------------------------------- launcher

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
    return cudaFuncSetAttribute(k_blk_rfused<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)blk_rgemm_smem(split));
}

cudaError_t blk_gj_sweep(const SysDesc *d_sys, const std::vector<SysDesc> &h_sys, int max_m, int max_ncol,
                         float2 *ws, int split, BlkScratch &scr, Status *st, int stage, cudaStream_t s, KTimer &kt) {
    const int nsys = (int)h_sys.size();
    cudaError_t e = cudaSuccess;
    BLK_SPLIT_DISPATCH(split, (e = set_blk_attrs<SS>(split)));
    if (e != cudaSuccess) return e;
    const size_t fsm = blk_factor_smem(split), rsm = blk_rgemm_smem(split);
    for (int k = 0; k < max_m; k += NBK) {
        double fl_fac = 0, fl_r = 0, fl_upd = 0;
        for (const SysDesc &S : h_sys) {
            if (k >= S.m) continue;
            double nbe = std::min(NBK, S.m - k), cols = S.ncol - k - nbe;
            fl_fac += 2.0 * nbe * nbe * nbe;
            fl_r += 2.0 * nbe * nbe * cols;
            fl_upd += 2.0 * (S.m - nbe) * nbe * cols;
        }
        const int cols = max_ncol - k;
        const int cb = (cols + 63) / 64, rb = (max_m + 127) / 128;
        kt.begin(GM_K_PANEL, fl_fac, s);
        BLK_SPLIT_DISPATCH(split, (k_blk_factor<SS><<<nsys, FAC_THREADS, fsm, s>>>(
                                      d_sys, ws, k, scr.x_dig, scr.a11_dig, scr.inv_plane, scr.x_ex, scr.a11_ex,
                                      scr.pmag, st, stage)));
        kt.end(s);
        kt.begin(GM_K_PIVROWS, fl_r, s);
        BLK_SPLIT_DISPATCH(split, (k_blk_rfused<SS><<<dim3(cb + rb, nsys), 128, rsm, s>>>(
                                      d_sys, ws, k, cb, scr.x_dig, scr.a11_dig, scr.inv_plane, scr.x_ex, scr.a11_ex,
                                      scr.fdig, scr.fplane, scr.fex, scr.rdig, scr.cplane, scr.rex, scr.pmag,
                                      st)));
        kt.end(s);
        kt.begin(GM_K_GJUPDATE, fl_upd, s);
        BLK_SPLIT_DISPATCH(split, (k_blk_update<SS><<<dim3((max_m + 63) / 64, (cols + 63) / 64, nsys), 128, 0, s>>>(
                                      d_sys, ws, k, scr.fdig, scr.fplane, scr.fex, scr.rdig, scr.cplane, scr.rex)));
        kt.end(s);
    }
    return cudaGetLastError();
}

}  // namespace gm
