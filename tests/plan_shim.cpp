// Test-only shim: builds the library's host plan (quad-tree, rings, P1..P4 tables,
// arena and workspace offsets) with the library's own plan.cpp and writes it out as a
// flat int64 record, so that CPU tests can check it against the oracle's tree.  Compiled
// by the tests with g++ together with plan.cpp; no CUDA involved.
//
// Record layout (all int64):
//   rc, L, leaf_doubles, arena_doubles, coef_total, nleaves, nstages, nroots
//   per root:  n, r, off, coef, problem
//   per leaf:  x0, y0, a, b, off, n, prob, coef
//   per stage: orient, nmerges, out_base, out_doubles, ws_doubles, dig_elems, exp_elems,
//              max_m, max_ncol, max_rp
//     per merge: s1, s2, out, ws, r1, r2, rp, sp, n1, n2, orient, n, kpad, eoff, doff, prob,
//                child1 (x0, y0, a, b), child2 (...), parent (...),
//                then the index table: p3[sp] p4[sp] g3[sp] g4[sp] p1[n1] q1[n1] p2[n2]
//                q2[n2] x12[8]
#include <cstdint>
#include <vector>

#include "../paper_1302_5995_gb300/csrc/gm_internal.h"

namespace {

void put_plan(const gm::Plan &P, int rc, std::vector<int64_t> &o) {
    o.insert(o.end(), {rc, P.L, P.leaf_doubles, P.arena_doubles, P.coef_total, (int64_t)P.leaves.size(),
                       (int64_t)P.stages.size(), (int64_t)P.roots.size()});
    for (const gm::RootDesc &r : P.roots) o.insert(o.end(), {r.n, r.r, r.off, r.coef, r.problem});
    for (const gm::LeafDesc &l : P.leaves) o.insert(o.end(), {l.x0, l.y0, l.a, l.b, l.off, l.n, l.prob, l.coef});
    for (const gm::Stage &st : P.stages) {
        o.insert(o.end(), {st.orient, (int64_t)st.merges.size(), st.out_base, st.out_doubles, st.ws_doubles,
                           st.dig_elems, st.exp_elems, st.max_m, st.max_ncol, st.max_rp});
        for (size_t k = 0; k < st.merges.size(); ++k) {
            const gm::MergeDesc &m = st.merges[k];
            o.insert(o.end(), {m.s1, m.s2, m.out, m.ws, m.r1, m.r2, m.rp, m.sp, m.n1, m.n2, m.orient, m.n, m.kpad,
                               m.eoff, m.doff, m.prob});
            for (const gm::Box &b : {st.in_boxes[2 * k], st.in_boxes[2 * k + 1], st.out_boxes[k]})
                o.insert(o.end(), {b.x0, b.y0, b.a, b.b});
            const int len = 4 * m.sp + 2 * m.n1 + 2 * m.n2 + 8;
            const int *t = st.table.data() + m.tab;
            o.insert(o.end(), t, t + len);
        }
    }
}

int64_t emit(const std::vector<int64_t> &o, int64_t *buf, int64_t cap) {
    if ((int64_t)o.size() > cap) return -(int64_t)o.size();
    for (size_t i = 0; i < o.size(); ++i) buf[i] = o[i];
    return (int64_t)o.size();
}

}  // namespace

extern "C" {

// One problem's plan.  Returns the record length, or -(needed length) if cap is short.
int64_t plan_dump(int n, int leaf, int64_t *buf, int64_t cap) {
    gm::Plan P;
    int rc = gm::build_plan(n, leaf, P);
    std::vector<int64_t> o;
    put_plan(P, rc, o);
    return emit(o, buf, cap);
}

// The batched plan of `count` problems (sizes ns, leaves, coefficient offsets coef).
int64_t plan_dump_batch(int count, const int *ns, const int *leaves, const int64_t *coef, int64_t *buf,
                        int64_t cap) {
    std::vector<gm::Plan> plans(count);
    std::vector<const gm::Plan *> ptr;
    std::vector<int64_t> off;
    for (int i = 0; i < count; ++i) {
        int rc = gm::build_plan(ns[i], leaves[i], plans[i]);
        if (rc) {
            std::vector<int64_t> o{rc};
            return emit(o, buf, cap);
        }
        ptr.push_back(&plans[i]);
        off.push_back(coef[i]);
    }
    gm::Plan B;
    int rc = gm::build_batch_plan(ptr, off, B);
    std::vector<int64_t> o;
    put_plan(B, rc, o);
    return emit(o, buf, cap);
}

}  // extern "C"
