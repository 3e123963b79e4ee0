"""The arithmetic scheme of the split-digit products, emulated on the CPU in numpy (no GPU
code involved): 6-bit truncated digits relative to each row's / column's largest entry,
digit pairs s + t <= S + 1 grouped by level L = s + t into units whose exact integer sums
stay within 2^24 (so an FP32 accumulator holds them exactly), and the error bound the GPU
tests use.  A mistake in the unit lengths or the pair selection shows here first."""
import numpy as np
import pytest

S = 9
BITS = 6
BK = 64
CHUNK = 4096


def level_blocks(L):
    """k blocks per unit of level L: (L - 1) pairs, digit products up to 63^2."""
    return min((1 << 24) // ((L - 1) * 3969 * BK), CHUNK // BK)


def digits(X, axis):
    """Row (axis=1) or column (axis=0) exponents and S signed 6-bit digits (truncation)."""
    m = np.max(np.abs(X), axis=axis, keepdims=True)
    e = np.where(m > 0, np.floor(np.log2(np.where(m > 0, m, 1.0))) + 1, 0.0).astype(int)
    r = np.ldexp(X, -e)
    q = np.trunc(np.ldexp(np.abs(r), BITS * S)).astype(np.int64)
    sg = np.sign(r)
    out = [sg * ((q >> (BITS * (S - 1 - s))) & 63) for s in range(S)]
    return e, out


def split_product(A, B):
    """A @ B the way the kernel forms it: per level and unit an exact integer sum, then
    scaled by 2^-6L into an FP64 accumulator."""
    K = A.shape[1]
    ea, Ad = digits(A, 1)
    eb, Bd = digits(B, 0)
    kblocks = (K + BK - 1) // BK
    acc = np.zeros((A.shape[0], B.shape[1]))
    for L in range(2, S + 2):
        cb = level_blocks(L)
        for c0 in range(0, kblocks, cb):
            k0, k1 = c0 * BK, min(K, (c0 + cb) * BK)
            unit = np.zeros_like(acc)
            for s in range(1, L):
                t = L - s
                unit += Ad[s - 1][:, k0:k1] @ Bd[t - 1][k0:k1, :]
            assert np.abs(unit).max() <= 2 ** 24  # exact in the FP32 accumulator
            acc += np.ldexp(unit, -BITS * L)
    return np.ldexp(np.ldexp(acc, ea), eb)


def bound(A, B, K):
    aA, aB = np.abs(A), np.abs(B)
    rowmax, colmax = aA.max(axis=1, keepdims=True), aB.max(axis=0, keepdims=True)
    return (S + 2) * K * 2.0 ** (-BITS * S) * (2 * rowmax) * (2 * colmax) + 2 * K * 2.0 ** -53 * (aA @ aB)


def test_unit_lengths_keep_sums_exact():
    for L in range(2, S + 2):
        cb = level_blocks(L)
        assert cb >= 1 and (L - 1) * 63 * 63 * cb * BK <= 2 ** 24
    assert [level_blocks(L) for L in (2, 10)] == [64, 7]


def test_digits_reconstruct_to_54_bits():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((20, 30)) * 10.0 ** rng.uniform(-5, 5, (20, 1))
    e, D = digits(X, 1)
    rec = sum(np.ldexp(D[s], -BITS * (s + 1)) for s in range(S))
    assert np.all(np.abs(np.ldexp(rec, e) - X) <= np.ldexp(np.ones_like(X), e - BITS * S))
    assert all(np.abs(d).max() <= 63 for d in D)


@pytest.mark.parametrize("scaling", ["plain", "ill"])
@pytest.mark.parametrize("shape", [(33, 40, 700), (17, 9, 4500)])
def test_split_product_within_bound(scaling, shape):
    M, N, K = shape
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    if scaling == "ill":
        A = A * 10.0 ** rng.uniform(-8, 8, (M, 1)) * 10.0 ** rng.uniform(-3, 3, A.shape)
        B = B * 10.0 ** rng.uniform(-8, 8, (1, N)) * 10.0 ** rng.uniform(-3, 3, B.shape)
    C = split_product(A, B)
    exact = A.astype(np.longdouble) @ B.astype(np.longdouble)
    assert np.all(np.abs(C - exact) <= bound(A, B, K))


def test_saturated_digits_reach_the_limit_and_stay_exact():
    x = 1.0 - 2.0 ** -52
    K = 4160
    A = np.full((3, K), x)
    B = np.full((K, 2), x)
    C = split_product(A, B)
    assert np.all(np.abs(C - K * x * x) <= bound(A, B, K))
