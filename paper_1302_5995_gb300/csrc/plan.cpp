// Host plan builder: the quad-tree (Section 2), ring orders, and the P1..P4 index
// tables of every pairwise merge (Section 3.2, eq. partition_we), grouped into one
// stage per (level, merge direction) in the order of Section 3.3.
#include <algorithm>
#include <map>
#include <tuple>

#include "gm_internal.h"

namespace gm {

namespace {

using Key = std::tuple<int, int, int, int>;
Key key(const Box &b) { return Key(b.x0, b.y0, b.a, b.b); }

void children(const Box &p, Box out[4]) {
    int a0 = p.a / 2, b0 = p.b / 2;  // west / south halves take the floor
    out[0] = {p.x0, p.y0, a0, b0};
    out[1] = {p.x0 + a0, p.y0, p.a - a0, b0};
    out[2] = {p.x0, p.y0 + b0, a0, p.b - b0};
    out[3] = {p.x0 + a0, p.y0 + b0, p.a - a0, p.b - b0};
}

int num_levels(int n, int leaf) {
    int L = 0;
    while ((n + (1 << L) - 1) / (1 << L) > leaf) ++L;
    return L;
}

// Append the merge of c1 (west/south) and c2 (east/north) into parent to the stage.
void add_merge(Stage &st, int n, const Box &c1, int64_t s1, const Box &c2, int64_t s2, const Box &par,
               int64_t out, int64_t &ws) {
    MergeDesc m{};
    m.s1 = s1;
    m.s2 = s2;
    m.out = out;
    m.r1 = ring_size(c1.a, c1.b);
    m.r2 = ring_size(c2.a, c2.b);
    m.rp = ring_size(par.a, par.b);
    m.orient = st.orient;
    m.n = n;
    std::vector<int> p3, p4, g3, g4, p1, q1, p2, q2;
    auto gidx = [n](int x, int y) { return x + n * y; };
    if (st.orient == 0) {  // shared vertical edge: child 1's east column, child 2's west column
        for (int j = 1; j < c1.b - 1; ++j) {
            p3.push_back(ring_pos(c1.a, c1.b, c1.a - 1, j));
            g3.push_back(gidx(c1.x0 + c1.a - 1, c1.y0 + j));
            p4.push_back(ring_pos(c2.a, c2.b, 0, j));
            g4.push_back(gidx(c2.x0, c2.y0 + j));
        }
    } else {  // shared horizontal edge: child 1's north row, child 2's south row
        for (int i = 1; i < c1.a - 1; ++i) {
            p3.push_back(ring_pos(c1.a, c1.b, i, c1.b - 1));
            g3.push_back(gidx(c1.x0 + i, c1.y0 + c1.b - 1));
            p4.push_back(ring_pos(c2.a, c2.b, i, 0));
            g4.push_back(gidx(c2.x0 + i, c2.y0));
        }
    }
    m.sp = (int)p3.size();
    // P1 / P2: the children's ring nodes that lie on the parent's ring, in ring order
    auto collect = [&](const Box &c, std::vector<int> &pk, std::vector<int> &qk) {
        int r = ring_size(c.a, c.b);
        std::vector<int> pos_of(r, -1);
        for (int j = 0; j < c.b; ++j)
            for (int i = 0; i < c.a; ++i) {
                int p = ring_pos(c.a, c.b, i, j);
                if (p < 0) continue;
                int pi = c.x0 + i - par.x0, pj = c.y0 + j - par.y0;
                pos_of[p] = ring_pos(par.a, par.b, pi, pj);
            }
        for (int p = 0; p < r; ++p)
            if (pos_of[p] >= 0) {
                pk.push_back(p);
                qk.push_back(pos_of[p]);
            }
    };
    collect(c1, p1, q1);
    collect(c2, p2, q2);
    m.n1 = (int)p1.size();
    m.n2 = (int)p2.size();
    // the two corner couplings across the shared edge (A12 / A21)
    int x12[8];
    for (int e = 0; e < 2; ++e) {
        int i1, j1, i2, j2;
        if (st.orient == 0) {
            i1 = c1.a - 1; j1 = e ? c1.b - 1 : 0; i2 = 0; j2 = j1;
        } else {
            i1 = e ? c1.a - 1 : 0; j1 = c1.b - 1; i2 = i1; j2 = 0;
        }
        int rp1 = ring_pos(c1.a, c1.b, i1, j1), rp2 = ring_pos(c2.a, c2.b, i2, j2);
        int a1 = (int)(std::find(p1.begin(), p1.end(), rp1) - p1.begin());
        int a2 = (int)(std::find(p2.begin(), p2.end(), rp2) - p2.begin());
        x12[4 * e + 0] = a1;
        x12[4 * e + 1] = a2;
        x12[4 * e + 2] = gidx(c1.x0 + i1, c1.y0 + j1);
        x12[4 * e + 3] = gidx(c2.x0 + i2, c2.y0 + j2);
    }
    m.tab = (int)st.table.size();
    auto app = [&](const std::vector<int> &v) { st.table.insert(st.table.end(), v.begin(), v.end()); };
    app(p3); app(p4); app(g3); app(g4); app(p1); app(q1); app(p2); app(q2);
    st.table.insert(st.table.end(), x12, x12 + 8);
    int mm = 2 * m.sp, ncol = mm + m.rp;
    m.ws = ws;
    ws += (int64_t)mm * ncol;
    m.kpad = (mm + 15) / 16 * 16;
    if (m.kpad == 0) m.kpad = 16;
    m.doff = st.dig_elems;
    st.dig_elems += (int64_t)((m.rp + 127) / 128 * 128) * m.kpad;  // rows padded to 128-row tiles
    m.eoff = (int)st.exp_elems;
    st.exp_elems += m.rp;
    st.max_m = std::max(st.max_m, mm);
    st.max_ncol = std::max(st.max_ncol, ncol);
    st.max_rp = std::max(st.max_rp, m.rp);
    st.merges.push_back(m);
    st.in_boxes.push_back(c1);
    st.in_boxes.push_back(c2);
    st.out_boxes.push_back(par);
}

}  // namespace

int build_plan(int n, int leaf, Plan &plan) {
    if (n < 2 || leaf < 3) return GM_EINVAL;
    plan = Plan{};
    plan.n = n;
    plan.leaf = leaf;
    // Leaves wider than the leaf kernels take (edge 17) are eliminated in nested-dissection
    // order: the tree continues below the requested leaf level with boxes of edge <= 16.
    // The splits are the same at every level, so the requested leaves are the boxes of
    // level L_user of this tree, and their Schur complements are exact eliminations.
    plan.L_user = num_levels(n, leaf);
    plan.L = num_levels(n, leaf <= kMaxLeafEdge ? leaf : 16);
    std::vector<std::vector<Box>> levels(plan.L + 1);
    levels[0].push_back({0, 0, n, n});
    for (int l = 0; l < plan.L; ++l)
        for (const Box &p : levels[l]) {
            Box c[4];
            children(p, c);
            for (int k = 0; k < 4; ++k) levels[l + 1].push_back(c[k]);
        }
    // leaves
    std::map<Key, int64_t> off;
    int64_t acc = 0;
    for (const Box &b : levels[plan.L]) {
        if (b.a < 2 || b.b < 2) return GM_EINVAL;
        LeafDesc d{b.x0, b.y0, b.a, b.b, acc, n, 0, 0};
        off[key(b)] = acc;
        int r = ring_size(b.a, b.b);
        acc += (int64_t)r * r;
        plan.leaves.push_back(d);
        plan.leaf_boxes.push_back(b);
    }
    plan.leaf_doubles = acc;
    // merge stages, finest level first; per level: horizontal, then vertical.  Each stage
    // writes the next region of the single arena.
    int64_t base = acc;
    for (int l = plan.L; l >= 1; --l) {
        Stage H{}, V{};
        H.orient = 0;
        V.orient = 1;
        std::map<Key, int64_t> half_off, par_off;
        int64_t hacc = base, hws = 0, vws = 0;
        for (const Box &p : levels[l - 1]) {
            Box c[4];
            children(p, c);
            Box south{p.x0, p.y0, p.a, c[0].b}, north{p.x0, p.y0 + c[0].b, p.a, c[2].b};
            half_off[key(south)] = hacc;
            add_merge(H, n, c[0], off.at(key(c[0])), c[1], off.at(key(c[1])), south, hacc, hws);
            hacc += (int64_t)ring_size(south.a, south.b) * ring_size(south.a, south.b);
            half_off[key(north)] = hacc;
            add_merge(H, n, c[2], off.at(key(c[2])), c[3], off.at(key(c[3])), north, hacc, hws);
            hacc += (int64_t)ring_size(north.a, north.b) * ring_size(north.a, north.b);
        }
        int64_t pacc = hacc;
        for (const Box &p : levels[l - 1]) {
            Box c[4];
            children(p, c);
            Box south{p.x0, p.y0, p.a, c[0].b}, north{p.x0, p.y0 + c[0].b, p.a, c[2].b};
            par_off[key(p)] = pacc;
            add_merge(V, n, south, half_off.at(key(south)), north, half_off.at(key(north)), p, pacc, vws);
            pacc += (int64_t)ring_size(p.a, p.b) * ring_size(p.a, p.b);
        }
        H.out_base = base;
        H.out_doubles = hacc - base;
        H.ws_doubles = hws;
        V.out_base = hacc;
        V.out_doubles = pacc - hacc;
        V.ws_doubles = vws;
        plan.stages.push_back(std::move(H));
        plan.stages.push_back(std::move(V));
        off = par_off;
        base = pacc;
    }
    plan.arena_doubles = base;
    plan.coef_total = (int64_t)n * n;
    plan.root = {0, 0, n, n};
    plan.r_root = ring_size(n, n);
    plan.roots.push_back(RootDesc{n, plan.r_root, off.at(key(plan.root)), 0, 0});
    return validate_plan(plan);
}

int build_batch_plan(const std::vector<const Plan *> &plans, const std::vector<int64_t> &coef_off, Plan &out) {
    out = Plan{};
    if (plans.empty() || plans.size() != coef_off.size()) return GM_EINVAL;
    int Lmax = 0;
    for (const Plan *p : plans) Lmax = std::max(Lmax, p->L);
    const int NS = 2 * Lmax;
    out.n = plans[0]->n;
    out.leaf = plans[0]->leaf;
    out.L = Lmax;
    out.L_user = 0;
    for (const Plan *p : plans) out.L_user = std::max(out.L_user, p->L_user);
    out.stages.resize(NS);
    for (int s = 0; s < NS; ++s) out.stages[s].orient = s % 2;
    // global layout: all leaves, then aligned stage 0 of all problems, stage 1, ...
    int64_t leaves_total = 0;
    std::vector<int64_t> stage_total(NS, 0);
    for (const Plan *p : plans) {
        leaves_total += p->leaf_doubles;
        const int shift = NS - 2 * p->L;
        for (size_t si = 0; si < p->stages.size(); ++si) stage_total[shift + si] += p->stages[si].out_doubles;
    }
    std::vector<int64_t> stage_base(NS, 0);
    int64_t acc = leaves_total;
    for (int s = 0; s < NS; ++s) {
        stage_base[s] = acc;
        acc += stage_total[s];
    }
    out.arena_doubles = acc;
    out.leaf_doubles = leaves_total;
    out.coef_total = 0;
    for (size_t pi = 0; pi < plans.size(); ++pi)
        out.coef_total = std::max(out.coef_total, coef_off[pi] + (int64_t)plans[pi]->n * plans[pi]->n);
    std::vector<int64_t> stage_fill(NS, 0), ws_fill(NS, 0);
    int64_t leaf_fill = 0;
    for (size_t pi = 0; pi < plans.size(); ++pi) {
        const Plan &P = *plans[pi];
        const int64_t co = coef_off[pi];
        const int shift = NS - 2 * P.L;
        // local arena regions of this problem and their global positions
        std::vector<std::pair<int64_t, int64_t>> lo_hi;  // local [begin, end)
        std::vector<int64_t> delta;
        lo_hi.push_back({0, P.leaf_doubles});
        delta.push_back(leaf_fill);
        for (size_t si = 0; si < P.stages.size(); ++si) {
            const Stage &st = P.stages[si];
            lo_hi.push_back({st.out_base, st.out_base + st.out_doubles});
            delta.push_back(stage_base[shift + si] + stage_fill[shift + si] - st.out_base);
        }
        auto remap = [&](int64_t x) -> int64_t {
            for (size_t q = 0; q < lo_hi.size(); ++q)
                if (x >= lo_hi[q].first && x < lo_hi[q].second) return x + delta[q];
            return -1;
        };
        for (const LeafDesc &l : P.leaves) {
            LeafDesc d = l;
            d.off = remap(l.off);
            d.coef = co;
            d.prob = (int)pi;
            out.leaves.push_back(d);
        }
        out.leaf_boxes.insert(out.leaf_boxes.end(), P.leaf_boxes.begin(), P.leaf_boxes.end());
        for (size_t si = 0; si < P.stages.size(); ++si) {
            const Stage &src = P.stages[si];
            Stage &dst = out.stages[shift + si];
            for (const MergeDesc &m0 : src.merges) {
                MergeDesc m = m0;
                m.s1 = remap(m0.s1);
                m.s2 = remap(m0.s2);
                m.out = remap(m0.out);
                m.ws = m0.ws + ws_fill[shift + si];
                m.prob = (int)pi;
                m.doff = dst.dig_elems;
                dst.dig_elems += (int64_t)((m.rp + 127) / 128 * 128) * m.kpad;
                m.eoff = (int)dst.exp_elems;
                dst.exp_elems += m.rp;
                const int *t = src.table.data() + m0.tab;
                const int len = 4 * m.sp + 2 * m.n1 + 2 * m.n2 + 8;
                std::vector<int> tab(t, t + len);
                for (int q = 2 * m.sp; q < 4 * m.sp; ++q) tab[q] += (int)co;
                int *x12 = tab.data() + 4 * m.sp + 2 * m.n1 + 2 * m.n2;
                x12[2] += (int)co;
                x12[3] += (int)co;
                x12[6] += (int)co;
                x12[7] += (int)co;
                m.tab = (int)dst.table.size();
                dst.table.insert(dst.table.end(), tab.begin(), tab.end());
                dst.merges.push_back(m);
                dst.max_m = std::max(dst.max_m, 2 * m.sp);
                dst.max_ncol = std::max(dst.max_ncol, 2 * m.sp + m.rp);
                dst.max_rp = std::max(dst.max_rp, m.rp);
            }
            dst.out_boxes.insert(dst.out_boxes.end(), src.out_boxes.begin(), src.out_boxes.end());
            dst.in_boxes.insert(dst.in_boxes.end(), src.in_boxes.begin(), src.in_boxes.end());
            stage_fill[shift + si] += src.out_doubles;
            ws_fill[shift + si] += src.ws_doubles;
        }
        RootDesc rd = P.roots[0];
        rd.off = remap(rd.off);
        rd.coef = co;
        rd.problem = (int)pi;
        out.roots.push_back(rd);
        leaf_fill += P.leaf_doubles;
    }
    for (int s = 0; s < NS; ++s) {
        out.stages[s].out_base = stage_base[s];
        out.stages[s].out_doubles = stage_total[s];
        out.stages[s].ws_doubles = ws_fill[s];
    }
    out.r_root = 0;
    for (const RootDesc &r : out.roots) out.r_root = std::max(out.r_root, r.r);
    return validate_plan(out);
}

// Every gather/scatter index of every stage stays inside its matrix, the parent
// positions of P1 and P2 form a permutation of the parent ring, and every S block lies
// inside its arena.
int validate_plan(const Plan &plan) {
    const int64_t NC = plan.coef_total;
    if (plan.coef_total > 0x7fffffff) return GM_EUNSUPPORTED;  // node indices are 32-bit
    for (const RootDesc &r : plan.roots)
        if (r.off < 0 || r.off + (int64_t)r.r * r.r > plan.arena_doubles || r.r != 4 * r.n - 4) return GM_EINVAL;
    for (const LeafDesc &d : plan.leaves) {
        int r = ring_size(d.a, d.b);
        if (d.off < 0 || d.off + (int64_t)r * r > plan.leaf_doubles) return GM_EINVAL;
        if (d.x0 < 0 || d.y0 < 0 || d.x0 + d.a > d.n || d.y0 + d.b > d.n) return GM_EINVAL;
    }
    for (const Stage &st : plan.stages) {
        for (const MergeDesc &m : st.merges) {
            if (m.n1 + m.sp != m.r1 || m.n2 + m.sp != m.r2 || m.n1 + m.n2 != m.rp) return GM_EINVAL;
            if (m.s1 < 0 || m.s1 + (int64_t)m.r1 * m.r1 > st.out_base) return GM_EINVAL;
            if (m.s2 < 0 || m.s2 + (int64_t)m.r2 * m.r2 > st.out_base) return GM_EINVAL;
            if (m.out < st.out_base || m.out + (int64_t)m.rp * m.rp > st.out_base + st.out_doubles) return GM_EINVAL;
            int mm = 2 * m.sp;
            if (m.ws < 0 || m.ws + (int64_t)mm * (mm + m.rp) > st.ws_doubles) return GM_EINVAL;
            if (m.kpad < mm || m.kpad % 16 || m.doff < 0 || m.doff % 2048 ||
                m.doff + (int64_t)((m.rp + 127) / 128 * 128) * m.kpad > st.dig_elems)
                return GM_EINVAL;
            if (m.eoff < 0 || m.eoff + m.rp > st.exp_elems) return GM_EINVAL;
            const int *t = st.table.data() + m.tab;
            if (m.tab + 4 * m.sp + 2 * m.n1 + 2 * m.n2 + 8 > (int)st.table.size()) return GM_EINVAL;
            const int *p3 = t, *p4 = t + m.sp, *g3 = t + 2 * m.sp, *g4 = t + 3 * m.sp;
            const int *p1 = t + 4 * m.sp, *q1 = p1 + m.n1, *p2 = q1 + m.n1, *q2 = p2 + m.n2;
            const int *x12 = q2 + m.n2;
            for (int k = 0; k < m.sp; ++k) {
                if (p3[k] < 0 || p3[k] >= m.r1 || p4[k] < 0 || p4[k] >= m.r2) return GM_EINVAL;
                if (g3[k] < 0 || g3[k] >= NC || g4[k] < 0 || g4[k] >= NC) return GM_EINVAL;
            }
            std::vector<char> seen(m.rp, 0);
            for (int k = 0; k < m.n1; ++k) {
                if (p1[k] < 0 || p1[k] >= m.r1 || q1[k] < 0 || q1[k] >= m.rp || seen[q1[k]]) return GM_EINVAL;
                seen[q1[k]] = 1;
            }
            for (int k = 0; k < m.n2; ++k) {
                if (p2[k] < 0 || p2[k] >= m.r2 || q2[k] < 0 || q2[k] >= m.rp || seen[q2[k]]) return GM_EINVAL;
                seen[q2[k]] = 1;
            }
            for (int e = 0; e < 2; ++e) {
                if (x12[4 * e] < 0 || x12[4 * e] >= m.n1 || x12[4 * e + 1] < 0 || x12[4 * e + 1] >= m.n2)
                    return GM_EINVAL;
                if (x12[4 * e + 2] < 0 || x12[4 * e + 2] >= NC || x12[4 * e + 3] < 0 ||
                    x12[4 * e + 3] >= NC)
                    return GM_EINVAL;
            }
        }
    }
    return GM_OK;
}

}  // namespace gm
