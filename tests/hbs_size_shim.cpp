// Test-only shim: the library's count of a root operator in HBS form
// (csrc/hbs_size.cpp) for a tree given as node ranges and ranks (nodes 1 .. 2^(L+1) - 1,
// arrays indexed by node, entry 0 unused).  Host code only.
#include <cstdint>

#include "../paper_1302_5995_gb300/csrc/hbs.h"

extern "C" int64_t hbs_size(int L, const int *lo, const int *hi, const int *k) {
    gm::HbsRoot h;
    h.L = L;
    const int NN = 1 << (L + 1);
    h.lo.assign(lo, lo + NN);
    h.hi.assign(hi, hi + NN);
    h.k.assign(k, k + NN);
    return gm::hbs_operator_doubles(h);
}
