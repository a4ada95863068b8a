// Internal structures shared by the host plan builder and the CUDA kernels.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/gm.h"

namespace gm {

// A rectangle of unknowns [x0, x0+a) x [y0, y0+b).
struct Box {
    int x0, y0, a, b;
};

inline int ring_size(int a, int b) { return 2 * a + 2 * b - 4; }

// Position of local node (i, j) on the ring of an a x b box (counter-clockwise from the
// south-west corner), or -1 for an interior node.
inline int ring_pos(int a, int b, int i, int j) {
    if (j == 0) return i;
    if (i == a - 1) return a - 1 + j;
    if (j == b - 1) return (a - 1) + (b - 1) + (a - 1 - i);
    if (i == 0) return 2 * (a - 1) + (b - 1) + (b - 1 - j);
    return -1;
}

// Direction codes of the five-point stencil weights.
enum { DIR_C = 0, DIR_E = 1, DIR_W = 2, DIR_N = 3, DIR_S = 4 };

// One leaf elimination.
struct LeafDesc {
    int x0, y0, a, b;
    int64_t off;   // S offset (doubles) in the output arena, column-major r x r
    int n;         // grid size of the leaf's problem (h = 1/(n+1))
    int prob;      // problem index in the batch (selects its Status)
    int64_t coef;  // offset of the problem's coefficients in the b, c, d arrays
};

// One pairwise merge (eq. S_fromtwo_nd).  Child 1 is west/south, child 2 east/north.
// All Schur complements of a build live in one arena; offsets are absolute in it.
struct MergeDesc {
    int64_t s1, s2;  // child Schur complements (arena offsets)
    int64_t out;     // parent Schur complement (arena offset)
    int64_t ws;      // dense system [M | Z] (workspace offset), column-major, ld = 2*sp
    int r1, r2, rp;  // ring sizes
    int sp;          // |P3| = |P4| (interface nodes of each child)
    int n1, n2;      // |P1|, |P2|; n1 + n2 = rp
    int orient;      // 0: child 2 east of child 1; 1: child 2 north of child 1
    int n;           // grid size of the merge's problem (h = 1/(n+1)); the table's global
                     // node indices already include the problem's coefficient offset
    int tab;         // offset of this merge's index table (ints)
    int kpad;        // 2*sp rounded up to 16 (row length of this merge's digit planes)
    int eoff;        // first row of this merge in the stage's exponent vectors (prefix of rp)
    int prob;        // problem index in the batch
    int64_t doff;    // first element of this merge in the stage's digit planes (rp x kpad)
    // table layout at tab:
    //   p3[sp]  p4[sp]  g3[sp]  g4[sp]         ring positions / global flat indices
    //   p1[n1]  q1[n1]  p2[n2]  q2[n2]         child ring positions / parent ring positions
    //   x12[8]: (a1, c1, g1, g2) x 2           P1-index, P2-index, global indices of the
    //                                           two corner couplings across the shared edge
};

// One dense system handled by the Gauss-Jordan sweep: [M | Z], m x ncol, column-major.
struct SysDesc {
    int64_t off;  // workspace offset (doubles)
    int m;        // order of M (columns eliminated)
    int ncol;     // m + number of right-hand-side columns
    int id;       // stage-local id for error reports
    int roff;     // first row of this system in per-stage row scratch (prefix sum of m)
    int coff;     // first column of this system in per-stage column scratch (prefix of ncol)
    int prob;     // problem index in the batch (selects its Status)
};

// Device status written by kernels, one per problem of a build.
struct Status {
    int code;                    // 0 or GM_ESINGULAR
    int where;                   // stage index of the first failure
    unsigned long long min_piv;  // bit pattern of min |pivot| (positive double)
    int growth;                  // block pivoting: a row outside a block would have pivoted
    unsigned int rho;            // block pivoting: largest refinement ratio |X0 E| / |R| of a
                                 // block solve (float bits; ordered like the values)
};

// One merge stage (all horizontal merges of a level, or all vertical ones).
struct Stage {
    int orient;
    std::vector<MergeDesc> merges;
    std::vector<int> table;
    std::vector<Box> in_boxes, out_boxes;  // per merge: child1, child2 / parent
    int64_t out_base;     // first arena element of this stage's outputs
    int64_t out_doubles;  // arena elements written by this stage
    int64_t ws_doubles;   // workspace elements of this stage
    int64_t dig_elems;  // elements of one digit plane of the stage (sum of rp * kpad)
    int64_t exp_elems;  // rows of the stage's exponent vectors (sum of rp)
    int max_m, max_ncol, max_rp;
};

// Root of one problem of a (possibly batched) plan.
struct RootDesc {
    int n, r;        // grid size, root ring size 4n - 4
    int64_t off;     // S_root offset in the last level's arena
    int64_t coef;    // offset of the problem's coefficients
    int problem;     // index in the batch
};

// Launch-shape choices of a build that the autotuner may change (the defaults were the
// fastest measured on the 512^2 convection workload).
struct Tune {
    int rtile32_max = 96;  // R kernel: 32-column tiles while systems x 64-column tiles <= this
    int tc_min_k = 192;    // merge update on tcgen05 for interfaces with K >= this (else mma.sync)
    int early = 0;         // blocked sweep: the early-factor schedule (next factor off the R chain)
    int a11 = 0;           // blocked sweep: only the next diagonal tile on the chain before its factor
    int upd_tiles = 0;     // blocked sweep's bulk update: 64-column tiles per CTA (0 one wave, -1 one per CTA)
};

// Largest leaf edge the leaf kernels take (band and inner-ring solves in shared memory).
constexpr int kMaxLeafEdge = 17;

struct Plan {
    int n, leaf, L;
    int L_user;  // levels of the tree for the requested leaf (L is larger when leaf > kMaxLeafEdge)
    std::vector<RootDesc> roots;
    std::vector<LeafDesc> leaves;
    std::vector<Box> leaf_boxes;
    int64_t leaf_doubles;   // leaves occupy arena elements [0, leaf_doubles)
    int64_t arena_doubles;  // every Schur complement of the build
    int64_t coef_total;     // length of each of the b, c, d arrays (all problems)
    std::vector<Stage> stages;  // 2 per level, finest first: H(L), V(L), H(L-1), ...
    Box root;
    int r_root;
};

int build_plan(int n, int leaf, Plan &plan);
// Concatenate the plans of several problems; stages are aligned from the root, so a
// problem with fewer levels has no merges in the finest stages of the batch.
int build_batch_plan(const std::vector<const Plan *> &plans, const std::vector<int64_t> &coef_off, Plan &out);

// The dense DtN matrix of a handle and its grid size (nullptr for a NULL handle).
const double *handle_dtn(gm_handle *h, int *n);
// For a mixed-precision handle: the digit planes of T's rows (bf16), their exponents
// and the digits per operand, as the split-product apply reads them; false otherwise.
bool handle_split(gm_handle *h, const void **tdig, const int **tex, int *split);
// True when [a, a + n) and [b, b + n) (doubles) share an element.
inline bool overlaps(const double *a, const double *b, size_t n) { return a < b + n && b < a + n; }
int validate_plan(const Plan &plan);

}  // namespace gm
