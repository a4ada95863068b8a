// HBS root: the root Schur complement compressed to the paper's HBS form (Section 4),
// inverted by Algorithm 1 (Section 5) and applied by Algorithm 2 in the solve stage.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gm_internal.h"
#include "kernels.h"

namespace gm {

constexpr int HBS_SAMPLES = 128;  // random samples per compression (columns of Omega, Psi)
constexpr int HBS_KCAP = 96;      // largest rank a node may take (oversampling >= 32)

struct HbsRoot {
    int r = 0, n = 0, m = 0, L = 0;
    double tol = 0.0;
    std::vector<int> lo, hi, k;  // per node 1 .. 2^(L+1) - 1: index range [lo, hi), rank
    double *pool = nullptr;      // every factor (cudaMalloc, owned)
    int64_t pool_doubles = 0;
    std::vector<int64_t> offE, offFt, offG;  // Algorithm 1 factors per node (pool offsets)
    int64_t offG1 = 0;                       // root G_1 = [G_1-system | inverse], q = k_2 + k_3
    int64_t offKK = 0, offWW = 0;            // ghost couplings of the ring (2 ints, 2 doubles per node)
    int max_rank = 0;
};

// Compress S (r x r FP64, column-major, device) at relative tolerance tol with node size
// m (2 <= m <= 192), run Algorithm 1, and tabulate the ghost couplings of the ring from
// b, c, d (n x n each).  GM_EUNSUPPORTED: a node's rank reached HBS_KCAP, or r <= m.
int hbs_build_root(const double *S, int r, int n, int m, double tol, const double *bf, const double *cf,
                   const double *df, cudaStream_t s, HbsRoot &out);
// dudn = (g - P S^{-1} B g)/h for B vectors (g, dudn: 4n x B column-major, device),
// S^{-1} applied by Algorithm 2.
int hbs_apply_dtn(HbsRoot &h, const double *g, double *dudn, int B, cudaStream_t s);
// The dense 4n x 4n DtN matrix of an HBS root (the solve applied to the identity);
// T may be host or device memory.
int hbs_dense_dtn(HbsRoot &h, double *T, cudaStream_t s);
cudaError_t hbs_df32_to_f64(const float2 *x, double *y, int64_t cnt, cudaStream_t s);
void hbs_free(HbsRoot &h);

}  // namespace gm
