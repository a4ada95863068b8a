// Body loads at listed nodes (Section 6.3): the second operator F of v = T g + F f_hat.
//
// Every box carries, beside its Schur complement S, a load map L (ring x m, column-major,
// m = the body nodes inside the box): at a leaf L = E_b - A_bi A_ii^{-1} E_i (Section
// 3.1, the right-hand side left on the ring after eliminating the interior), at a merge
// the updated right-hand side of Section 3.2 applied to the children's maps,
//     L = [L1(P1) 0; 0 L2(P2)] - [S13 0; 0 S24] [S33 A34; A43 S44]^{-1} [L1(P3) 0; 0 L2(P4)],
// whose last factor is solved with the merge's own interface system as extra columns of
// Z; at the root S_root u = B g + L f_hat, so F = -P S_root^{-1} L / h.  A box's columns
// are its first child's, then its second child's; a leaf's follow the caller's list.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "gm_internal.h"
#include "kernels.h"

namespace gm {

// A leaf that holds body nodes.
struct LeafLoadDesc {
    int x0, y0, a, b;  // the leaf box
    int n;             // grid size
    int m;             // body nodes inside it
    int col0;          // first entry of its nodes in LoadPlan::leaf_nodes
    int ni;            // interior nodes (a-2)(b-2)
    int64_t sys;       // its system [A_ii | E_i] (ni x (ni + m)) in the leaf workspace, or -1 if ni = 0
    int64_t lout;      // its load map (ring x m) in the load arena
};

// A merge's load columns, beside the plan's MergeDesc (same order within a stage).
struct MergeLoadDesc {
    int m1, m2;        // columns of child 1 and child 2
    int64_t l1, l2;    // children's load maps in the load arena (-1 when m = 0)
    int64_t lout;      // the parent's load map (-1 when m1 + m2 = 0)
    int64_t ws;        // this merge's system [M | Z | Z_L] in the stage's load workspace
};

struct LoadPlan {
    int nbody = 0;
    std::vector<LeafLoadDesc> leaves;
    std::vector<int> leaf_nodes;      // per leaf with loads: its body nodes (flat i + n j), concatenated
    std::vector<SysDesc> leaf_sys;    // the leaves' [A_ii | E_i] systems for the dense sweep
    int64_t leaf_ws = 0;              // doubles of those systems
    int leaf_max_m = 0, leaf_max_ncol = 0;
    std::vector<std::vector<MergeLoadDesc>> stages;  // per plan stage, per merge
    std::vector<std::vector<MergeDesc>> merges;      // the plan's merges with ws moved to the load layout
    std::vector<std::vector<SysDesc>> sys;           // their systems, ncol = 2 sp + rp + m1 + m2
    std::vector<int64_t> stage_ws;                   // doubles of each stage's load workspace
    std::vector<int> stage_max_ncol;
    int64_t arena = 0;                // doubles of the load arena (every box's load map)
    int64_t root_l = -1;              // the root's load map (ring x nbody)
    std::vector<int> root_order;      // root column c holds the body node at caller position root_order[c]
};

// Builds the load plan of a single-problem plan for body nodes `body` (flat i + n j,
// distinct, inside the grid).  GM_EINVAL for a bad list, a batched plan or nbody = 0.
int build_load_plan(const Plan &plan, const std::vector<int> &body, LoadPlan &lp);

// Kernels (loads.cu).
cudaError_t launch_leaf_load_assemble(const LeafLoadDesc *d, int nl, const int *nodes, double *ws, int max_elems,
                                      const double *b, const double *c, const double *dd, cudaStream_t s);
cudaError_t launch_leaf_load_finalize(const LeafLoadDesc *d, int nl, const int *nodes, const double *ws,
                                      double *larena, int max_rm, const double *b, const double *c,
                                      const double *dd, cudaStream_t s);
cudaError_t launch_merge_load_assemble(const MergeDesc *md, const MergeLoadDesc *ld, int nm, const int *tab,
                                       const double *larena, double *ws, int64_t max_elems, cudaStream_t s);
cudaError_t launch_merge_load_update(const MergeDesc *md, const MergeLoadDesc *ld, int nm, const int *tab,
                                     const double *in, const double *ws, double *larena, int64_t max_elems,
                                     cudaStream_t s);
cudaError_t launch_load_finalize(const double *xl, int r, int n, int m, const int *order, double *F, cudaStream_t s);
cudaError_t launch_apply_add(const double *F, const double *Fl, double *V, int N, int m, int B, cudaStream_t s);

}  // namespace gm
