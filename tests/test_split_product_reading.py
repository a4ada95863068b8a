"""Reading of the mixed-precision products (exact split products on the tensor cores):
each operand row is scaled by a power of two and cut into S signed 7-bit digits
(|d| <= 64, exact in bf16); the digit-pair products of equal level g = a + b are summed in
FP32, which is exact while the level sum stays below 2^24: level g holds g + 1 pairs of at
most K products of 64 x 64, so K <= 512 keeps every level of S <= 6 exact; the levels
recombine to the product with a relative error near 2^-7S.  Checked in numpy: the FP32
level sums equal the exact integer sums, the recombined product meets the bound for
S = 4 and 6, and the worst case fits 2^24 at K = 512 but not at K = 2048.
"""
import numpy as np
import pytest


def digits(X, S):
    """Rows of X -> (S digit planes, row exponents e): X ~ sum_s d_s 2^(e - 6 - 7 s)."""
    mx = np.abs(X).max(axis=1)
    e = np.where(mx > 0, np.frexp(mx * (1 + 1e-7))[1], 0)
    t = X * np.exp2(6.0 - e)[:, None]
    out = []
    for _ in range(S):
        d = np.rint(t)
        out.append(d)
        t = (t - d) * 128.0
    return np.array(out), e


def split_product(A, B, S):
    """A B^T from digit-pair level sums accumulated in FP32."""
    dA, ea = digits(A, S)
    dB, eb = digits(B, S)
    levels, exact = [], []
    for g in range(S):
        acc32 = np.zeros((A.shape[0], B.shape[0]), np.float32)
        acc64 = np.zeros((A.shape[0], B.shape[0]))
        for a in range(g + 1):
            p = dA[a].astype(np.float32) @ dB[g - a].T.astype(np.float32)  # FP32 accumulation
            acc32 += p
            acc64 += dA[a] @ dB[g - a].T
        levels.append(acc32)
        exact.append(acc64)
    val = sum(levels[g].astype(np.float64) * 2.0 ** (-7 * g) for g in range(S))
    return val * np.exp2(ea[:, None] + eb[None, :] - 12.0), levels, exact


@pytest.mark.parametrize("S,bound", [(4, 2.0 ** -24), (6, 2.0 ** -38)])
def test_split_product_is_exact_per_level_and_accurate(S, bound):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((24, 512)) * np.exp2(rng.integers(-8, 8, (24, 1)))
    B = rng.standard_normal((16, 512))
    P, levels, exact = split_product(A, B, S)
    for g in range(S):
        assert np.array_equal(levels[g].astype(np.float64), exact[g])
        assert np.abs(exact[g]).max() < 2.0 ** 24
    ref = A @ B.T
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * A.shape[1]
    assert (np.abs(P - ref) / scale).max() < bound


def test_level_sums_need_the_k_chunk_bound():
    # worst case: every digit at the extreme |d| = 64 and all signs aligned; level g sums
    # g + 1 digit pairs of K products each
    worst = lambda g, K: (g + 1) * K * 64 * 64
    assert all(worst(g, 512) < 2 ** 24 for g in range(6))  # the chunk every kernel uses
    assert worst(5, 2048) >= 2 ** 24                        # a 2048 chunk would not be exact
    # and FP32 really does round such a sum: one step past 2^24 loses the unit
    acc = np.float32(2 ** 24)
    assert acc + np.float32(1) == acc


def test_merged_low_levels_stay_below_the_truncation():
    """A reading for wider tensor-memory tiles: levels 0..2 stay exact in their own FP32
    accumulators, levels 3..5 share one.  Their products come from copies of the digit
    planes scaled by powers of two, A'_a = d_a 2^-7a and B'_b = d_b 2^(21 - 7b), so each
    product d_a d_b 2^-7(a+b-3) carries its level's factor exactly (bf16 holds any 7-bit
    digit times a power of two), and only the shared FP32 sum rounds -- near 2^-24 of
    level 3, i.e. 2^-45 of the product, below the 2^-42 truncation of S = 6 digits."""
    S, K = 6, 512
    rng = np.random.default_rng(11)
    A = rng.standard_normal((32, K)) * np.exp2(rng.integers(-6, 6, (32, 1)))
    B = rng.standard_normal((24, K))
    dA, ea = digits(A, S)
    dB, eb = digits(B, S)
    exact_levels = []
    for g in range(3):
        acc = np.zeros((A.shape[0], B.shape[0]), np.float32)
        for a in range(g + 1):
            acc += dA[a].astype(np.float32) @ dB[g - a].T.astype(np.float32)
        exact_levels.append(acc.astype(np.float64))
    Ap = np.stack([dA[a] * 2.0 ** (-7 * a) for a in range(S)]).astype(np.float32)
    Bp = np.stack([dB[b] * 2.0 ** (21 - 7 * b) for b in range(S)]).astype(np.float32)
    merged = np.zeros((A.shape[0], B.shape[0]), np.float32)
    for a in range(S):
        for b in range(S):
            if 3 <= a + b <= S - 1:
                merged += Ap[a] @ Bp[b].T  # FP32 products of exact operands, FP32 sum
    val = sum(exact_levels[g] * 2.0 ** (-7 * g) for g in range(3)) + merged.astype(np.float64) * 2.0 ** -21
    P = val * np.exp2(ea[:, None] + eb[None, :] - 12.0)
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * K
    assert (np.abs(P - A @ B.T) / scale).max() < 2.0 ** -38
    # the same bound as six exact levels
    P6, _, _ = split_product(A, B, S)
    assert (np.abs(P - A @ B.T) / scale).max() < 4 * (np.abs(P6 - A @ B.T) / scale).max() + 2.0 ** -44


def _two_sum32(a, b):
    s = (a + b).astype(np.float32)
    bb = (s - a).astype(np.float32)
    e = ((a - (s - bb)).astype(np.float32) + (b - bb).astype(np.float32)).astype(np.float32)
    return s, e


def _df_add_f32(hi, lo, b):
    """(hi, lo) + b in double-float: FP32 two-sum, then the low parts, renormalised."""
    s, e = _two_sum32(hi, b)
    e = (e + lo).astype(np.float32)
    h = (s + e).astype(np.float32)
    return h, (e - (h - s)).astype(np.float32)


def test_recombination_with_the_low_levels_summed_in_fp32():
    """The bulk update's recombination of the six exact level sums: levels 5, 4, 3 added in
    plain FP32 (scaled by 2^-35, 2^-28, 2^-21: roundings near 2^-24 of level 3), then
    levels 2, 1, 0 added in double-float.  Against the exact recombination in FP64 the
    error stays below 2^-47 of the product bound |A| |B| K (64 x 64 x K in digit units),
    far under the 2^-42 truncation of S = 6 digits; with level 2 also in plain FP32 it
    would reach that truncation."""
    S, K = 6, 512
    rng = np.random.default_rng(12)
    A = rng.standard_normal((32, K)) * np.exp2(rng.integers(-6, 6, (32, 1)))
    B = rng.standard_normal((24, K))
    _, levels, exact = split_product(A, B, S)
    lv = [lvl.astype(np.float32) for lvl in levels]
    ref = sum(exact[g] * 2.0 ** (-7 * g) for g in range(S))
    scale = 64.0 * 64.0 * K  # the product bound in digit units

    def combine(n_plain):
        lo = np.zeros_like(lv[0])
        for g in range(S - 1, S - 1 - n_plain, -1):
            lo = (lo + lv[g] * np.float32(2.0 ** (-7 * g))).astype(np.float32)
        hi, lo2 = lo, np.zeros_like(lo)
        for g in range(S - 1 - n_plain, -1, -1):
            hi, lo2 = _df_add_f32(hi, lo2, (lv[g] * np.float32(2.0 ** (-7 * g))).astype(np.float32))
        return hi.astype(np.float64) + lo2.astype(np.float64)

    assert np.abs(combine(3) - ref).max() < 2.0 ** -47 * scale
    assert np.abs(combine(1) - ref).max() < 2.0 ** -47 * scale   # all six in double-float
    assert np.abs(combine(4) - ref).max() > 2.0 ** -45 * scale   # level 2 too: near the truncation
