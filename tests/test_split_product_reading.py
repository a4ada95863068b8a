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
