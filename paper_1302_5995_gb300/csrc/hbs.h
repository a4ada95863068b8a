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
    double *sig = nullptr;  // conductance networks: the ghosts' link conductivities (4n, owned), which
                            // weight the rows of every apply (the datum is the link current)
};

// HBS factors of a dense r x r FP64 matrix S (column-major, leading dimension lds,
// device): compression at relative tolerance tol with node size m (Section 4), then
// Algorithm 1 (Section 5).  GM_EUNSUPPORTED: a node's rank reached HBS_KCAP, or r <= m.
int hbs_factor(const double *S, int lds, int r, int m, double tol, cudaStream_t s, HbsRoot &out);
// Y = S^{-1} X for B columns (Algorithm 2); X, Y device, r x B, leading dimensions ldx, ldy.
int hbs_solve(HbsRoot &h, const double *X, int ldx, double *Y, int ldy, int B, cudaStream_t s);

// The interface solve of a pairwise merge by the paper's accelerated Step 1: X = M^{-1} Z
// for M = [S33 A34; A43 S44] by block elimination with HBS inverses of S33 and of its
// Schur complement T44 = S44 - A43 S33^{-1} A34 (A34, A43 diagonal):
//   [V3 W3] = S33^{-1} [A34 Z3],  X4 = T44^{-1} (Z4 - A43 W3),  X3 = W3 - V3 X4.
// ws is the merge's dense system [M | Z] (2 sp rows, ld 2 sp, 2 sp + rp columns); on
// success its right block holds X, as after the dense elimination; on failure (e.g.
// GM_EUNSUPPORTED) ws is unchanged.  max_rank (optional) accumulates the largest rank.
int hbs_block_solve(double *ws, int sp, int rp, int m, double tol, cudaStream_t s, int *max_rank);

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
// Doubles of the operator in HBS form (Section 4), from the node ranks: D, U, V of every
// leaf, U, V of every inner node below the root, and the two B blocks between the
// children of every inner node -- the memory the paper reports as M(n).
int64_t hbs_operator_doubles(const HbsRoot &h);

}  // namespace gm
