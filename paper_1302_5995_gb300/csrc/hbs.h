// HBS root: the root Schur complement compressed to the paper's HBS form (Section 4),
// inverted by Algorithm 1 (Section 5) and applied by Algorithm 2 in the solve stage.
#pragma once
#include <map>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gm_internal.h"
#include "kernels.h"

namespace gm {

constexpr int HBS_SAMPLES = 128;      // random samples per node at the first attempt (columns of
                                      // Omega, Psi); doubled while a rank comes within
constexpr int HBS_OVERSAMPLE = 32;    // this many of the sample count,
constexpr int HBS_MAX_SAMPLES = 512;  // up to this many samples: ranks up to 480
constexpr int HBS_MARGIN = 32;        // QR columns kept past a basis' own truncation point
// Largest relative residual max |S S^{-1} x - x| / max |x| accepted from Algorithm 1's
// inverse (checked on four Gaussian vectors after every factorisation); beyond it the
// inverse is unstable and the factorisation returns GM_EUNSUPPORTED.
constexpr double HBS_MAX_RESIDUAL = 1e-3;
// Returned (not a public code) by hbs_factor, hbs_build_root and hbs_block_solve when the
// residual check fails: the caller eliminates that system densely instead.
constexpr int HBS_UNSTABLE = 1001;

struct HbsRoot {
    int r = 0, n = 0, m = 0, L = 0;
    double tol = 0.0;
    std::vector<int> lo, hi, k;  // per node 1 .. 2^(L+1) - 1: index range [lo, hi), rank
    double *pool = nullptr;      // the inverse's factors E, F^T, G, G_1 and the ghost couplings (owned)
    cudaStream_t pool_stream = nullptr;  // non-null: pool is a stream-ordered temporary
    int64_t pool_doubles = 0;
    std::vector<int64_t> offE, offFt, offG;  // Algorithm 1 factors per node (pool offsets)
    int64_t offG1 = 0;                       // root G_1 = [G_1-system | inverse], q = k_2 + k_3
    int64_t offKK = 0, offWW = 0;            // ghost couplings of the ring (2 ints, 2 doubles per node)
    int max_rank = 0;
    int max_trunc = 0;      // largest truncation point of a node's samples (sets the sample count)
    double residual = 0.0;  // relative residual of the inverse on random vectors (see hbs_factor)
    double *sig = nullptr;  // conductance networks: the ghosts' link conductivities (4n, owned), which
                            // weight the rows of every apply (the datum is the link current)
};

// HBS factors of a dense r x r FP64 matrix S (column-major, leading dimension lds,
// device): compression at relative tolerance tol with node size m (Section 4), then
// Algorithm 1 (Section 5).  The compression's temporaries come from the library pool;
// the inverse's factors from cudaMalloc, or (temp) from the pool on stream s.
// GM_EUNSUPPORTED: a node's rank exceeds HBS_MAX_SAMPLES - HBS_OVERSAMPLE, a sample has
// more rows than one factorisation takes, or r <= m.  HBS_UNSTABLE: the inverse failed
// the residual check (HBS_MAX_RESIDUAL).
int hbs_factor(const double *S, int lds, int r, int m, double tol, cudaStream_t s, HbsRoot &out, bool temp);
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

// Steps 2 and 3 of the accelerated merge (Section 5) for one merge whose interface
// system was solved (X = M^{-1} Z in the right block of ws, the merge's [M | Z], ld 2 sp):
// S13 = S1(P1, P3) and S24 = S2(P2, P4) are compressed to L13 R13, L24 R24 at relative
// tolerance tol (from Gaussian samples), the update is formed as [L13 (R13 X3);
// L24 (R24 X4)], and the parent's Schur complement [S11 A12; A21 S22] minus it is written
// densely into its ring order at out + hm.out.  d_md: this merge's descriptor on the
// device; max_rank (optional) accumulates the larger of the two ranks.
int hbs_merge_lowrank(const MergeDesc &hm, const MergeDesc *d_md, const int *d_tab, const double *in,
                      const double *ws, double *out, const double *bf, const double *cf, const double *df, double tol,
                      cudaStream_t s, KTimer &kt, int *max_rank);

// Compress S (r x r FP64, column-major, device) at relative tolerance tol with node size
// m (2 <= m <= 192), run Algorithm 1, and tabulate the ghost couplings of the ring from
// b, c, d (n x n each).  GM_EUNSUPPORTED as for hbs_factor.
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
// A (rows x cols, column-major, ld rows, device) ~ L R at relative tolerance tol, from a
// Gaussian sample of A truncated at the first |R_jj| <= tol |R_11| of its pivoted QR: L
// (rows x k, orthonormal) and R = L^T A (k x cols) in new cudaMalloc buffers (owned by the
// caller), k in *k.
int hbs_lowrank(const double *A, int rows, int cols, double tol, cudaStream_t s, double **L, double **R, int *k);
// C (m x n) = alpha op(A) op(B) + beta C in FP64 (column-major; op(X) = X^T when tX).
int hbs_gemm(const double *A, int lda, int ta, const double *B, int ldb, int tb, double *C, int ldc, int m, int n,
             int k, double alpha, double beta, cudaStream_t s);
// Algorithmic flops of the HBS steps this thread issued since the last call (products,
// QR factorisations, dense inversions), then reset.
double hbs_flops_take();
// Factorisations run concurrently on several host threads (independent merges of a
// stage): hbs_hints_freeze() makes every sample-count lookup read the hints as they are
// now; a thread that calls hbs_hints_record(&m) writes its own hints into m instead of the
// shared table; hbs_hints_thaw(ms) merges the maps in order and ends the freeze.
void hbs_hints_freeze();
void hbs_hints_record(std::map<std::pair<int, int>, int> *out);
void hbs_hints_thaw(const std::vector<std::map<std::pair<int, int>, int>> &outs);
// Doubles of the operator in HBS form (Section 4), from the node ranks: D, U, V of every
// leaf, U, V of every inner node below the root, and the two B blocks between the
// children of every inner node -- the memory the paper reports as M(n).
int64_t hbs_operator_doubles(const HbsRoot &h);

}  // namespace gm
