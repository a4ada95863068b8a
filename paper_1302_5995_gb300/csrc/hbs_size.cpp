// Size of a root operator in HBS form (Section 4), from its node ranks: host code only.
#include "hbs.h"

namespace gm {

int64_t hbs_operator_doubles(const HbsRoot &h) {
    if (h.k.empty()) return 0;
    const int NN = 1 << (h.L + 1), first_leaf = 1 << h.L;
    int64_t tot = 0;
    for (int t = 1; t < NN; ++t) {
        const int64_t k = h.k[t];
        if (t >= first_leaf) {
            const int64_t p = h.hi[t] - h.lo[t];
            tot += p * p + 2 * p * k;  // D, U, V
        } else {
            const int64_t ka = h.k[2 * t], kb = h.k[2 * t + 1];
            tot += 2 * ka * kb;                   // B between the children
            if (t > 1) tot += 2 * (ka + kb) * k;  // U, V
        }
    }
    return tot;
}

}  // namespace gm
