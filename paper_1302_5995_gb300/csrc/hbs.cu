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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hbs.h"
#include "network.h"

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

// Basis of the column space of A (p x l, p <= QR_MAXP, l <= HBS_SAMPLES) by Gram-Schmidt
// with column pivoting: at step j the remaining column of largest norm is orthogonalised
// (twice) against Q(:, 0..j-1), normalised into Q(:, j) and removed from the others.
// out[0] = first j with |R_jj| <= tol |R_11| (or the steps taken), out[1] = columns of
// Q produced (stops at kmax or at a numerically zero column).
constexpr int QR_MAXP = 2 * HBS_KCAP;

struct QrDesc {
    const double *A;
    double *Q;
    int *out;
    int p, l, lda, ldq;
};

__global__ void __launch_bounds__(256) k_hbs_pqr(const QrDesc *__restrict__ ds, double tol, int kmax) {
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
    int ktr = -1, kval = 0;
    const int steps = min(kmax, min(p, l));
    for (int j = 0; j < steps; ++j) {
        // norms of the remaining columns, one warp per column
        for (int c = warp; c < l; c += nw) {
            double s = 0.0;
            if (!used[c])
                for (int i = lane; i < p; i += 32) s = fma(sA[(size_t)c * p + i], sA[(size_t)c * p + i], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) nrm[c] = used[c] ? -1.0 : s;
        }
        __syncthreads();
        if (tid == 0) {
            int pv = -1;
            double best = -1.0;
            for (int c = 0; c < l; ++c)
                if (nrm[c] > best) { best = nrm[c]; pv = c; }
            s_piv = pv;
            s_r = best > 0.0 ? sqrt(best) : 0.0;
            if (j == 0) s_r1 = s_r;
        }
        __syncthreads();
        const int pv = s_piv;
        const double rjj = s_r, r11 = s_r1;
        if (ktr < 0 && !(rjj > tol * r11)) ktr = j;
        if (pv < 0 || !(rjj > 1e-15 * r11) || !(r11 > 0.0)) break;
        for (int i = tid; i < p; i += blockDim.x) qv[i] = sA[(size_t)pv * p + i];
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {  // q -= Q (Q^T q), twice
            for (int c = warp; c < j; c += nw) {
                double s = 0.0;
                for (int i = lane; i < p; i += 32) s = fma(D.Q[i + (size_t)c * D.ldq], qv[i], s);
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) coef[c] = s;
            }
            __syncthreads();
            for (int i = tid; i < p; i += blockDim.x) {
                double v = qv[i];
                for (int c = 0; c < j; ++c) v = fma(-coef[c], D.Q[i + (size_t)c * D.ldq], v);
                qv[i] = v;
            }
            __syncthreads();
        }
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < p; i += 32) s = fma(qv[i], qv[i], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) s_r = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        }
        __syncthreads();
        const double inv = s_r;
        for (int i = tid; i < p; i += blockDim.x) {
            qv[i] *= inv;
            D.Q[i + (size_t)j * D.ldq] = qv[i];
        }
        if (tid == 0) used[pv] = 1;
        __syncthreads();
        // remove q from every remaining column
        for (int c = warp; c < l; c += nw) {
            if (used[c]) continue;
            double s = 0.0;
            for (int i = lane; i < p; i += 32) s = fma(qv[i], sA[(size_t)c * p + i], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            for (int i = lane; i < p; i += 32) sA[(size_t)c * p + i] = fma(-s, qv[i], sA[(size_t)c * p + i]);
        }
        __syncthreads();
        kval = j + 1;
    }
    if (tid == 0) {
        D.out[0] = ktr < 0 ? kval : ktr;
        D.out[1] = kval;
    }
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

int run_gemms(const std::vector<GemmDesc> &v, DescBuf &db, cudaStream_t s) {
    if (v.empty()) return GM_OK;
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
int invert_batch(const std::vector<std::pair<double *, int>> &mats, double *base, cudaStream_t s) {
    std::vector<SysDesc> h;
    int max_m = 0, roff = 0, coff = 0;
    for (size_t i = 0; i < mats.size(); ++i) {
        const int m = mats[i].second;
        if (m == 0) continue;
        h.push_back(SysDesc{(int64_t)(mats[i].first - base), m, 2 * m, (int)i, roff, coff, 0});
        roff += m;
        coff += 2 * m;
        max_m = std::max(max_m, m);
    }
    if (h.empty()) return GM_OK;
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

}  // namespace

int hbs_factor(const double *S, int lds, int r, int m, double tol, cudaStream_t s, HbsRoot &H) {
    if (r < 2 || lds < r || m < 2 || m > QR_MAXP || !(tol > 0.0)) return GM_EINVAL;
    const int l = HBS_SAMPLES, KC = HBS_KCAP;
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
    auto rows_bound = [&](int t) { return leaf(t) ? sz(t) : 2 * KC; };

    // ---- storage (upper bounds: a node's rank is at most KC)
    Bump bp;
    const int64_t oOm = bp.take((int64_t)r * l), oPs = bp.take((int64_t)r * l);
    const int64_t oY = bp.take((int64_t)r * l), oZ = bp.take((int64_t)r * l);
    const int64_t oKK = bp.take(r), oWW = bp.take(2 * (int64_t)r);  // coupling table (ints, doubles)
    std::vector<int64_t> oU(NN), oV(NN), oUf(NN), oVf(NN), oYs(NN), oZs(NN), oyr(NN), ozr(NN);
    std::vector<int64_t> oD(NN), oW(NN), oX(NN), oZt(NN);
    std::vector<int64_t> oHab(NN), oHba(NN), oWab(NN), oWba(NN), oXab(NN), oXba(NN);
    H.offE.assign(NN, 0);
    H.offFt.assign(NN, 0);
    H.offG.assign(NN, 0);
    for (int t = 2; t < NN; ++t) {
        const int rb = rows_bound(t);
        oU[t] = bp.take((int64_t)rb * KC);
        oV[t] = bp.take((int64_t)rb * KC);
        oUf[t] = leaf(t) ? oU[t] : bp.take((int64_t)sz(t) * KC);
        oVf[t] = leaf(t) ? oV[t] : bp.take((int64_t)sz(t) * KC);
        oYs[t] = bp.take((int64_t)rb * l);
        oZs[t] = bp.take((int64_t)rb * l);
        oyr[t] = bp.take((int64_t)KC * l);
        ozr[t] = bp.take((int64_t)KC * l);
        oD[t] = bp.take((int64_t)rb * 2 * rb);
        oW[t] = bp.take((int64_t)rb * KC);
        oX[t] = bp.take((int64_t)KC * 2 * KC);
        oZt[t] = bp.take((int64_t)KC * rb);
        H.offE[t] = bp.take((int64_t)rb * KC);
        H.offFt[t] = bp.take((int64_t)KC * rb);
        H.offG[t] = bp.take((int64_t)rb * rb);
    }
    for (int t = 1; t < (1 << L); ++t) {
        const int a = 2 * t, b = 2 * t + 1;
        oHab[t] = bp.take((int64_t)KC * KC);
        oHba[t] = bp.take((int64_t)KC * KC);
        oWab[t] = bp.take((int64_t)KC * sz(b));
        oWba[t] = bp.take((int64_t)KC * sz(a));
        oXab[t] = bp.take((int64_t)sz(a) * KC);
        oXba[t] = bp.take((int64_t)sz(b) * KC);
    }
    const int64_t oG1 = bp.take((int64_t)2 * KC * 4 * KC);
    const int64_t oOut = bp.take(2 * (int64_t)NN);  // QR results: 2 ints per node and kind (as doubles)
    const int64_t oOutV = bp.take(2 * (int64_t)NN);
    H.offG1 = oG1;
    H.pool_doubles = bp.top;
    if (cudaMalloc((void **)&H.pool, (size_t)bp.top * 8) != cudaSuccess) {
        cudaGetLastError();
        H.pool = nullptr;
        return GM_ENOMEM;
    }
    double *P = H.pool;
    int *outU = (int *)(P + oOut), *outV = (int *)(P + oOutV);
    DescBuf db;
    int rc;
    const size_t qr_smem = (size_t)QR_MAXP * l * sizeof(double);
    HCK(cudaFuncSetAttribute(k_hbs_pqr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qr_smem));

    // ---- samples Y = S Omega, Z = S^T Psi
    k_hbs_normals<<<256, 256, 0, s>>>(P + oOm, (int64_t)r * l, 0x4842530000000001ull);
    k_hbs_normals<<<256, 256, 0, s>>>(P + oPs, (int64_t)r * l, 0x4842530000000002ull);
    HCK(cudaGetLastError());
    if ((rc = run_gemms({gd(S, lds, 0, P + oOm, r, 0, P + oY, r, r, l, r, 1.0, 0.0),
                         gd(S, lds, 1, P + oPs, r, 0, P + oZ, r, r, l, r, 1.0, 0.0)},
                        db, s)))
        return rc;

    auto qr_level = [&](const std::vector<int> &nodes, const std::vector<int> &prow) -> int {
        std::vector<QrDesc> q;
        for (size_t i = 0; i < nodes.size(); ++i) {
            const int t = nodes[i], p = prow[i];
            q.push_back(QrDesc{P + oYs[t], P + oU[t], outU + 2 * t, p, l, p, p});
            q.push_back(QrDesc{P + oZs[t], P + oV[t], outV + 2 * t, p, l, p, p});
        }
        int rc2 = db.ensure(q.size() * sizeof(QrDesc), s);
        if (rc2) return rc2;
        HCK(cudaMemcpyAsync(db.p, q.data(), q.size() * sizeof(QrDesc), cudaMemcpyHostToDevice, s));
        k_hbs_pqr<<<(unsigned)q.size(), 256, qr_smem, s>>>((const QrDesc *)db.p, tol, KC);
        HCK(cudaGetLastError());
        std::vector<int> hu(2 * NN), hv(2 * NN);
        HCK(cudaMemcpyAsync(hu.data(), outU, 2 * NN * sizeof(int), cudaMemcpyDeviceToHost, s));
        HCK(cudaMemcpyAsync(hv.data(), outV, 2 * NN * sizeof(int), cudaMemcpyDeviceToHost, s));
        HCK(cudaStreamSynchronize(s));
        for (int t : nodes) {
            // one rank for U and V (Algorithm 1 inverts V* D^-1 U): the larger truncation
            // point, within the columns both factorisations produced
            int kt = std::max(hu[2 * t], hv[2 * t]);
            kt = std::min(kt, std::min(hu[2 * t + 1], hv[2 * t + 1]));
            if (kt >= KC) return GM_EUNSUPPORTED;
            H.k[t] = kt;
            H.max_rank = std::max(H.max_rank, kt);
        }
        return GM_OK;
    };

    // ---- leaves: sample of the off-diagonal block row / column, bases, reduced samples
    {
        std::vector<CopyDesc> cp;
        std::vector<GemmDesc> g;
        std::vector<int> nodes, prow;
        for (int t = 1 << L; t < NN; ++t) {
            const int lo = H.lo[t], p = sz(t);
            const double *Sd = S + lo + (size_t)lo * lds;
            cp.push_back(cpd(P + oY + lo, r, P + oYs[t], p, p, l, 0));
            cp.push_back(cpd(P + oZ + lo, r, P + oZs[t], p, p, l, 0));
            g.push_back(gd(Sd, lds, 0, P + oOm + lo, r, 0, P + oYs[t], p, p, l, p, -1.0, 1.0));
            g.push_back(gd(Sd, lds, 1, P + oPs + lo, r, 0, P + oZs[t], p, p, l, p, -1.0, 1.0));
            nodes.push_back(t);
            prow.push_back(p);
        }
        if ((rc = run_copies(cp, db, s)) || (rc = run_gemms(g, db, s)) || (rc = qr_level(nodes, prow))) return rc;
        g.clear();
        for (int t : nodes) {
            const int p = sz(t), k = H.k[t];
            g.push_back(gd(P + oU[t], p, 1, P + oYs[t], p, 0, P + oyr[t], std::max(k, 1), k, l, p, 1.0, 0.0));
            g.push_back(gd(P + oV[t], p, 1, P + oZs[t], p, 0, P + ozr[t], std::max(k, 1), k, l, p, 1.0, 0.0));
        }
        if ((rc = run_gemms(g, db, s))) return rc;
    }
    // ---- parents, finest first; the root (level 0) only needs its B blocks
    for (int lev = L - 1; lev >= 0; --lev) {
        std::vector<GemmDesc> g1, g2;
        std::vector<CopyDesc> cp;
        std::vector<int> nodes, prow;
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int a = 2 * t, b = 2 * t + 1, ka = H.k[a], kb = H.k[b];
            const int sa = sz(a), sb = sz(b);
            const double *Sab = S + H.lo[a] + (size_t)H.lo[b] * lds, *Sba = S + H.lo[b] + (size_t)H.lo[a] * lds;
            // W_ab = Uf_a^T S(I_a, I_b), W_ba = Uf_b^T S(I_b, I_a)
            g1.push_back(gd(P + oUf[a], sa, 1, Sab, lds, 0, P + oWab[t], std::max(ka, 1), ka, sb, sa, 1.0, 0.0));
            g1.push_back(gd(P + oUf[b], sb, 1, Sba, lds, 0, P + oWba[t], std::max(kb, 1), kb, sa, sb, 1.0, 0.0));
            // X_ab = S(I_a, I_b) Vf_b, X_ba = S(I_b, I_a) Vf_a
            g1.push_back(gd(Sab, lds, 0, P + oVf[b], sb, 0, P + oXab[t], sa, sa, kb, sb, 1.0, 0.0));
            g1.push_back(gd(Sba, lds, 0, P + oVf[a], sa, 0, P + oXba[t], sb, sb, ka, sa, 1.0, 0.0));
            // B_tau blocks: H_ab = W_ab Vf_b, H_ba = W_ba Vf_a
            g2.push_back(gd(P + oWab[t], std::max(ka, 1), 0, P + oVf[b], sb, 0, P + oHab[t], std::max(ka, 1), ka, kb,
                            sb, 1.0, 0.0));
            g2.push_back(gd(P + oWba[t], std::max(kb, 1), 0, P + oVf[a], sa, 0, P + oHba[t], std::max(kb, 1), kb, ka,
                            sa, 1.0, 0.0));
            if (lev >= 1) {
                const int p = ka + kb;
                // reduced samples: [y_a - W_ab Omega(I_b); y_b - W_ba Omega(I_a)], same for z
                cp.push_back(cpd(P + oyr[a], std::max(ka, 1), P + oYs[t], std::max(p, 1), ka, l, 0));
                cp.push_back(cpd(P + oyr[b], std::max(kb, 1), P + oYs[t] + ka, std::max(p, 1), kb, l, 0));
                cp.push_back(cpd(P + ozr[a], std::max(ka, 1), P + oZs[t], std::max(p, 1), ka, l, 0));
                cp.push_back(cpd(P + ozr[b], std::max(kb, 1), P + oZs[t] + ka, std::max(p, 1), kb, l, 0));
                g2.push_back(gd(P + oWab[t], std::max(ka, 1), 0, P + oOm + H.lo[b], r, 0, P + oYs[t], std::max(p, 1),
                                ka, l, sb, -1.0, 1.0));
                g2.push_back(gd(P + oWba[t], std::max(kb, 1), 0, P + oOm + H.lo[a], r, 0, P + oYs[t] + ka,
                                std::max(p, 1), kb, l, sa, -1.0, 1.0));
                g2.push_back(gd(P + oXba[t], sb, 1, P + oPs + H.lo[b], r, 0, P + oZs[t], std::max(p, 1), ka, l, sb,
                                -1.0, 1.0));
                g2.push_back(gd(P + oXab[t], sa, 1, P + oPs + H.lo[a], r, 0, P + oZs[t] + ka, std::max(p, 1), kb, l,
                                sa, -1.0, 1.0));
                nodes.push_back(t);
                prow.push_back(p);
            }
        }
        if ((rc = run_gemms(g1, db, s)) || (rc = run_copies(cp, db, s)) || (rc = run_gemms(g2, db, s))) return rc;
        if (lev == 0) break;
        if ((rc = qr_level(nodes, prow))) return rc;
        std::vector<GemmDesc> g3;
        for (int t : nodes) {
            const int a = 2 * t, b = 2 * t + 1, ka = H.k[a], kb = H.k[b], k = H.k[t], p = ka + kb;
            const int sa = sz(a), st = sz(t);
            g3.push_back(gd(P + oU[t], std::max(p, 1), 1, P + oYs[t], std::max(p, 1), 0, P + oyr[t], std::max(k, 1), k,
                            l, p, 1.0, 0.0));
            g3.push_back(gd(P + oV[t], std::max(p, 1), 1, P + oZs[t], std::max(p, 1), 0, P + ozr[t], std::max(k, 1), k,
                            l, p, 1.0, 0.0));
            // full bases: Uf_t = diag(Uf_a, Uf_b) U_t, likewise V
            g3.push_back(gd(P + oUf[a], sa, 0, P + oU[t], std::max(p, 1), 0, P + oUf[t], st, sa, k, ka, 1.0, 0.0));
            g3.push_back(gd(P + oUf[b], sz(b), 0, P + oU[t] + ka, std::max(p, 1), 0, P + oUf[t] + sa, st, sz(b), k, kb,
                            1.0, 0.0));
            g3.push_back(gd(P + oVf[a], sa, 0, P + oV[t], std::max(p, 1), 0, P + oVf[t], st, sa, k, ka, 1.0, 0.0));
            g3.push_back(gd(P + oVf[b], sz(b), 0, P + oV[t] + ka, std::max(p, 1), 0, P + oVf[t] + sa, st, sz(b), k, kb,
                            1.0, 0.0));
        }
        if ((rc = run_gemms(g3, db, s))) return rc;
    }

    // ---- Algorithm 1, finest level first
    auto rows_of = [&](int t) { return leaf(t) ? sz(t) : H.k[2 * t] + H.k[2 * t + 1]; };
    for (int lev = L; lev >= 1; --lev) {
        std::vector<CopyDesc> cp;
        std::vector<std::pair<double *, int>> inv;
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t);
            double *Dq = P + oD[t];  // [D~ | I], q x 2q, ld q
            if (leaf(t)) {
                cp.push_back(cpd(S + H.lo[t] + (size_t)H.lo[t] * lds, lds, Dq, q, q, q, 0));
            } else {
                const int a = 2 * t, b = 2 * t + 1, ka = H.k[a], kb = H.k[b];
                const double *Dha = P + oX[a] + (size_t)ka * ka, *Dhb = P + oX[b] + (size_t)kb * kb;
                cp.push_back(cpd(Dha, std::max(ka, 1), Dq, q, ka, ka, 0));
                cp.push_back(cpd(P + oHab[t], std::max(ka, 1), Dq + (size_t)ka * q, q, ka, kb, 0));
                cp.push_back(cpd(P + oHba[t], std::max(kb, 1), Dq + ka, q, kb, ka, 0));
                cp.push_back(cpd(Dhb, std::max(kb, 1), Dq + ka + (size_t)ka * q, q, kb, kb, 0));
            }
            cp.push_back(cpd(nullptr, 1, Dq + (size_t)q * q, q, q, q, 1));
            inv.push_back({Dq, q});
        }
        if ((rc = run_copies(cp, db, s)) || (rc = invert_batch(inv, P, s))) return rc;
        // W = D~^-1 U, X = V^T W (into [X | I]), then D^ = X^-1
        std::vector<GemmDesc> g;
        cp.clear();
        inv.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            const double *Di = P + oD[t] + (size_t)q * q;
            g.push_back(gd(Di, q, 0, P + oU[t], q, 0, P + oW[t], q, q, k, q, 1.0, 0.0));
            cp.push_back(cpd(nullptr, 1, P + oX[t] + (size_t)k * k, std::max(k, 1), k, k, 1));
            inv.push_back({P + oX[t], k});
        }
        if ((rc = run_gemms(g, db, s))) return rc;
        g.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            g.push_back(gd(P + oV[t], q, 1, P + oW[t], q, 0, P + oX[t], std::max(k, 1), k, k, q, 1.0, 0.0));
        }
        if ((rc = run_gemms(g, db, s)) || (rc = run_copies(cp, db, s)) || (rc = invert_batch(inv, P, s))) return rc;
        // E = W D^, Zt = V^T D~^-1, F^T = D^ Zt, G = D~^-1 - E Zt
        g.clear();
        cp.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            const double *Di = P + oD[t] + (size_t)q * q, *Dh = P + oX[t] + (size_t)k * k;
            g.push_back(gd(P + oW[t], q, 0, Dh, std::max(k, 1), 0, P + H.offE[t], q, q, k, k, 1.0, 0.0));
            g.push_back(gd(P + oV[t], q, 1, Di, q, 0, P + oZt[t], std::max(k, 1), k, q, q, 1.0, 0.0));
            cp.push_back(cpd(Di, q, P + H.offG[t], q, q, q, 0));
        }
        if ((rc = run_gemms(g, db, s)) || (rc = run_copies(cp, db, s))) return rc;
        g.clear();
        for (int t = 1 << lev; t < (2 << lev); ++t) {
            const int q = rows_of(t), k = H.k[t];
            const double *Dh = P + oX[t] + (size_t)k * k;
            g.push_back(gd(Dh, std::max(k, 1), 0, P + oZt[t], std::max(k, 1), 0, P + H.offFt[t], std::max(k, 1), k, q,
                           k, 1.0, 0.0));
            g.push_back(gd(P + H.offE[t], q, 0, P + oZt[t], std::max(k, 1), 0, P + H.offG[t], q, q, q, k, -1.0, 1.0));
        }
        if ((rc = run_gemms(g, db, s))) return rc;
    }
    // G_1 = [D^_2, B_23; B_32, D^_3]^{-1}
    {
        const int k2 = H.k[2], k3 = H.k[3], q = k2 + k3;
        double *Dq = P + oG1;
        std::vector<CopyDesc> cp{cpd(P + oX[2] + (size_t)k2 * k2, std::max(k2, 1), Dq, q, k2, k2, 0),
                                 cpd(P + oHab[1], std::max(k2, 1), Dq + (size_t)k2 * q, q, k2, k3, 0),
                                 cpd(P + oHba[1], std::max(k3, 1), Dq + k2, q, k3, k2, 0),
                                 cpd(P + oX[3] + (size_t)k3 * k3, std::max(k3, 1), Dq + k2 + (size_t)k2 * q, q, k3, k3, 0),
                                 cpd(nullptr, 1, Dq + (size_t)q * q, q, q, q, 1)};
        if ((rc = run_copies(cp, db, s)) || (rc = invert_batch({{Dq, q}}, P, s))) return rc;
    }
    H.offKK = oKK;
    H.offWW = oWW;
    HCK(cudaStreamSynchronize(s));
    return GM_OK;
}

int hbs_build_root(const double *S, int r, int n, int m, double tol, const double *bf, const double *cf,
                   const double *df, cudaStream_t s, HbsRoot &H) {
    int rc = hbs_factor(S, r, r, m, tol, s, H);
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
        if ((rc = hbs_factor(ws, M, sp, m, tol, s, H33))) break;
        // [V3 W3] = S33^{-1} [A34 Z3]: the columns sp .. of the top rows of [M | Z]
        if ((rc = hbs_solve(H33, ws + (size_t)sp * M, M, VW, sp, sp + rp, s))) break;
        // T44 = S44 - A43 V3, Z4' = Z4 - A43 W3 (A43 diagonal: M(sp + i, i))
        const int bx = (int)std::min<int64_t>(((int64_t)sp * std::max(sp, rp) + 255) / 256, 4096);
        k_hbs_sub_diag<<<bx, 256, 0, s>>>(T44, sp, ws + sp + (size_t)sp * M, M, ws + sp, M + 1, V3, sp, sp, sp);
        k_hbs_sub_diag<<<bx, 256, 0, s>>>(Z4, sp, ws + sp + (size_t)M * M, M, ws + sp, M + 1, W3, sp, sp, rp);
        if (cudaGetLastError() != cudaSuccess) { rc = GM_ECUDA; break; }
        if ((rc = hbs_factor(T44, sp, sp, m, tol, s, H44))) break;
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
    if (h.pool) cudaFree(h.pool);
    h.pool = nullptr;
    if (h.sig) cudaFree(h.sig);
    h.sig = nullptr;
}

}  // namespace gm
