// Test-only shim: builds the library's body-load plan (csrc/loads_plan.cpp) on top of its
// plain plan (csrc/plan.cpp) and writes it out as a flat int64 record for the CPU tests.
// No CUDA code runs; the CUDA headers are only needed for the declarations.
//
// Record: rc, nbody, arena, root_l, leaf_ws, nleaves, nstages, root_order[nbody],
//   per leaf: x0, y0, a, b, m, col0, ni, sys, lout, then its m body nodes
//   per leaf system: off, m, ncol, id
//   per stage: nmerges, stage_ws, max_ncol, then per merge:
//     m1, m2, l1, l2, lout, ws, sys.off, sys.m, sys.ncol, sys.id, copy_ok,
//     c1 (x0, y0, a, b), c2 (...), parent (...)
//   copy_ok: the merge descriptor copy differs from the plan's only in ws
#include <cstdint>
#include <cstring>
#include <vector>

#include "../paper_1302_5995_gb300/csrc/loads.h"

extern "C" int64_t load_plan_dump(int n, int leaf, const int *body, int nbody, int64_t *buf, int64_t cap) {
    gm::Plan P;
    std::vector<int64_t> o;
    int rc = gm::build_plan(n, leaf, P);
    gm::LoadPlan lp;
    if (!rc) rc = gm::build_load_plan(P, std::vector<int>(body, body + nbody), lp);
    o.insert(o.end(), {rc, lp.nbody, lp.arena, lp.root_l, lp.leaf_ws, (int64_t)lp.leaves.size(),
                       (int64_t)lp.stages.size()});
    if (!rc) {
        o.insert(o.end(), lp.root_order.begin(), lp.root_order.end());
        for (const gm::LeafLoadDesc &d : lp.leaves) {
            o.insert(o.end(), {d.x0, d.y0, d.a, d.b, d.m, d.col0, d.ni, d.sys, d.lout});
            o.insert(o.end(), lp.leaf_nodes.begin() + d.col0, lp.leaf_nodes.begin() + d.col0 + d.m);
        }
        for (const gm::SysDesc &s : lp.leaf_sys) o.insert(o.end(), {s.off, s.m, s.ncol, s.id});
        for (size_t si = 0; si < lp.stages.size(); ++si) {
            const gm::Stage &st = P.stages[si];
            o.insert(o.end(), {(int64_t)lp.stages[si].size(), lp.stage_ws[si], lp.stage_max_ncol[si]});
            for (size_t k = 0; k < lp.stages[si].size(); ++k) {
                const gm::MergeLoadDesc &d = lp.stages[si][k];
                const gm::SysDesc &s = lp.sys[si][k];
                gm::MergeDesc a = st.merges[k], b = lp.merges[si][k];
                const bool ws_ok = b.ws == d.ws;
                a.ws = b.ws = 0;
                const bool same = std::memcmp(&a, &b, sizeof a) == 0;
                o.insert(o.end(), {d.m1, d.m2, d.l1, d.l2, d.lout, d.ws, s.off, s.m, s.ncol, s.id,
                                   (int64_t)(ws_ok && same)});
                for (const gm::Box &bx : {st.in_boxes[2 * k], st.in_boxes[2 * k + 1], st.out_boxes[k]})
                    o.insert(o.end(), {bx.x0, bx.y0, bx.a, bx.b});
            }
        }
    }
    if ((int64_t)o.size() > cap) return -(int64_t)o.size();
    for (size_t i = 0; i < o.size(); ++i) buf[i] = o[i];
    return (int64_t)o.size();
}
