// Host plan of the body-load build (Section 6.3): which leaves hold body nodes, every
// box's load-map columns and their place in the load arena, and each merge's interface
// system widened by its children's load columns (in a workspace layout of its own, so
// the plain plan is untouched).
#include <algorithm>
#include <map>
#include <tuple>

#include "loads.h"

namespace gm {

namespace {

using Key = std::tuple<int, int, int, int>;
Key key(const Box &b) { return Key(b.x0, b.y0, b.a, b.b); }

struct BoxLoads {
    int64_t loff = -1;      // load map in the arena (-1: no loads inside)
    std::vector<int> cols;  // caller positions of its body nodes, in column order
};

}  // namespace

int build_load_plan(const Plan &P, const std::vector<int> &body, LoadPlan &lp) {
    lp = LoadPlan{};
    if (P.roots.size() != 1 || body.empty()) return GM_EINVAL;
    const int n = P.n;
    const int64_t N = (int64_t)n * n;
    std::vector<char> seen(N, 0);
    for (int g : body) {
        if (g < 0 || g >= N || seen[g]) return GM_EINVAL;
        seen[g] = 1;
    }
    lp.nbody = (int)body.size();
    std::map<Key, BoxLoads> boxes;
    int64_t acc = 0;  // load arena
    // leaves: their body nodes in the caller's order; [A_ii | E_i] when there is an interior
    int64_t wacc = 0;
    int roff = 0, coff = 0;
    for (const LeafDesc &l : P.leaves) {
        BoxLoads bl;
        for (int i = 0; i < (int)body.size(); ++i) {
            const int gx = body[i] % n, gy = body[i] / n;
            if (gx >= l.x0 && gx < l.x0 + l.a && gy >= l.y0 && gy < l.y0 + l.b) bl.cols.push_back(i);
        }
        if (!bl.cols.empty()) {
            LeafLoadDesc d{};
            d.x0 = l.x0;
            d.y0 = l.y0;
            d.a = l.a;
            d.b = l.b;
            d.n = n;
            d.m = (int)bl.cols.size();
            d.col0 = (int)lp.leaf_nodes.size();
            for (int c : bl.cols) lp.leaf_nodes.push_back(body[c]);
            d.ni = (l.a > 2 && l.b > 2) ? (l.a - 2) * (l.b - 2) : 0;
            d.sys = -1;
            if (d.ni > 0) {
                d.sys = wacc;
                SysDesc s{wacc, d.ni, d.ni + d.m, (int)lp.leaf_sys.size(), roff, coff, 0};
                roff += s.m;
                coff += s.ncol;
                wacc += (int64_t)s.m * s.ncol;
                lp.leaf_max_m = std::max(lp.leaf_max_m, s.m);
                lp.leaf_max_ncol = std::max(lp.leaf_max_ncol, s.ncol);
                lp.leaf_sys.push_back(s);
            }
            d.lout = acc;
            bl.loff = acc;
            acc += (int64_t)ring_size(l.a, l.b) * d.m;
            lp.leaves.push_back(d);
        }
        boxes[key(Box{l.x0, l.y0, l.a, l.b})] = bl;
    }
    lp.leaf_ws = wacc;
    // merges: child 1's columns, then child 2's
    for (const Stage &st : P.stages) {
        std::vector<MergeLoadDesc> L;
        std::vector<MergeDesc> M;
        std::vector<SysDesc> S;
        int64_t w = 0;
        int r0 = 0, c0 = 0, maxc = 0;
        for (size_t k = 0; k < st.merges.size(); ++k) {
            const MergeDesc &m = st.merges[k];
            auto f1 = boxes.find(key(st.in_boxes[2 * k])), f2 = boxes.find(key(st.in_boxes[2 * k + 1]));
            if (f1 == boxes.end() || f2 == boxes.end()) return GM_EINVAL;
            const BoxLoads &b1 = f1->second, &b2 = f2->second;
            MergeLoadDesc d{};
            d.m1 = (int)b1.cols.size();
            d.m2 = (int)b2.cols.size();
            d.l1 = b1.loff;
            d.l2 = b2.loff;
            BoxLoads bp;
            bp.cols = b1.cols;
            bp.cols.insert(bp.cols.end(), b2.cols.begin(), b2.cols.end());
            d.lout = -1;
            if (!bp.cols.empty()) {
                d.lout = acc;
                bp.loff = acc;
                acc += (int64_t)m.rp * (int64_t)bp.cols.size();
            }
            const int mm = 2 * m.sp, ncol = mm + m.rp + d.m1 + d.m2;
            d.ws = w;
            MergeDesc mc = m;
            mc.ws = w;
            S.push_back(SysDesc{w, mm, ncol, (int)k, r0, c0, 0});
            r0 += mm;
            c0 += ncol;
            w += (int64_t)mm * ncol;
            maxc = std::max(maxc, ncol);
            L.push_back(d);
            M.push_back(mc);
            boxes[key(st.out_boxes[k])] = bp;
        }
        lp.stages.push_back(std::move(L));
        lp.merges.push_back(std::move(M));
        lp.sys.push_back(std::move(S));
        lp.stage_ws.push_back(w);
        lp.stage_max_ncol.push_back(maxc);
    }
    lp.arena = acc;
    auto fr = boxes.find(key(P.root));
    if (fr == boxes.end() || (int)fr->second.cols.size() != lp.nbody) return GM_EINVAL;
    lp.root_l = fr->second.loff;
    lp.root_order = fr->second.cols;
    return GM_OK;
}

}  // namespace gm
