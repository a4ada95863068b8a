// Kernels of the conductance-network build (Section 6.1): the five-point weight table
// from the link conductivities, and the datum weights of the root operators.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gm_internal.h"
#include "network.h"

namespace gm {

__global__ void __launch_bounds__(256)
k_net_weights(const double *__restrict__ sx, const double *__restrict__ sy, int n, double *__restrict__ W,
              double *__restrict__ sig) {
    const double ih = n + 1.0, ih2 = ih * ih;
    const int64_t N2 = (int64_t)n * n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N2 + 4 * n;
         g += (int64_t)gridDim.x * blockDim.x) {
        if (g < N2) {
            const int i = (int)(g % n), j = (int)(g / n);
            const double e = sx[(i + 1) + (int64_t)(n + 1) * j], w = sx[i + (int64_t)(n + 1) * j];
            const double no = sy[i + (int64_t)n * (j + 1)], so = sy[i + (int64_t)n * j];
            double *o = W + 5 * g;
            o[DIR_C] = (e + w + no + so) * ih2;
            o[DIR_E] = -e * ih2;
            o[DIR_W] = -w * ih2;
            o[DIR_N] = -no * ih2;
            o[DIR_S] = -so * ih2;
        } else {  // ghost k: the link to its unknown neighbour
            const int k = (int)(g - N2), side = k / n, t = k % n;
            double v;
            if (side == 0) v = sy[t];                                   // south, below (t, 0)
            else if (side == 1) v = sx[n + (int64_t)(n + 1) * t];       // east, right of (n-1, t)
            else if (side == 2) v = sy[(n - 1 - t) + (int64_t)n * n];   // north, above (n-1-t, n-1)
            else v = sx[(int64_t)(n + 1) * (n - 1 - t)];                // west, left of (0, n-1-t)
            sig[k] = v;
        }
    }
}

__global__ void __launch_bounds__(256)
k_scale_rows(double *__restrict__ T, int N, int ncols, const double *__restrict__ sig) {
    const int64_t tot = (int64_t)N * ncols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        T[e] *= sig[e % N];
}

cudaError_t launch_net_weights(const double *sx, const double *sy, int n, double *W, double *sig, cudaStream_t s) {
    const int64_t tot = (int64_t)n * n + 4 * n;
    const int g = (int)std::min<int64_t>((tot + 255) / 256, 8192);
    k_net_weights<<<g, 256, 0, s>>>(sx, sy, n, W, sig);
    return cudaGetLastError();
}

cudaError_t launch_scale_rows(double *T, int N, int ncols, const double *sig, cudaStream_t s) {
    const int64_t tot = (int64_t)N * ncols;
    if (tot == 0) return cudaSuccess;
    const int g = (int)std::min<int64_t>((tot + 255) / 256, 8192);
    k_scale_rows<<<g, 256, 0, s>>>(T, N, ncols, sig);
    return cudaGetLastError();
}

}  // namespace gm
