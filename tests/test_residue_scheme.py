"""The number format of the residue form of the split products, restated on the CPU with
Python integers and exact rationals (no GPU code involved): operands truncated to p-bit
integers, their symmetric residues modulo 16 pairwise coprime moduli up to 256 (exact bf16
integers), exact FP32 sums over 1024-long k chunks, the chunk fold x - m round(x/m) in FP32
arithmetic, the weighted residues t_l = (X mod m_l) y_l mod m_l, and the Chinese-remainder
reconstruction with its quotient estimate from the top 32-bit limbs.  A wrong modulus, plan
size, fold, weight or quotient bound shows here first."""
from fractions import Fraction
from math import gcd, prod

import numpy as np
import pytest

# 2^8, 3*5*17, 11*23, 251, 13*19, 241, 239, 233, 229, 227, 223, 7*31, 211, 199, 197, 193
MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]
BK, CHUNK_BLOCKS = 64, 16
MAGIC = Fraction(3, 2) * 2 ** 23


def plan(Kp, bits=54):
    """Fewest moduli n with 2 Kp 2^{2p} <= M for some p >= bits (p as large as M allows,
    at most 62); None when 16 moduli fall short."""
    M = 1
    for n, m in enumerate(MODULI, 1):
        M *= m
        room = M // (2 * Kp)
        p = min((room.bit_length() - 1) // 2, 62) if room else -1
        if p >= bits:
            return n, p, M
    return None


def sym(x, m):
    """Symmetric residue of x modulo m, in (-m/2, m/2] (m even: +m/2 kept)."""
    r = x % m
    return r - m if 2 * r > m else r


def rn32(v):
    """v rounded to the nearest FP32 value (ties to even), as an exact rational."""
    v = Fraction(v)
    if v == 0:
        return Fraction(0)
    s, a = (1, v) if v > 0 else (-1, -v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    q, rem = divmod(a / ulp, 1)
    n = int(q)
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return s * n * ulp


def fold32(x, m):
    """The epilogue's fold in FP32: q = (x inv + 1.5 2^23) - 1.5 2^23 with one rounding for
    the fused multiply-add, then x - q m (exact)."""
    inv = rn32(Fraction(1, m))
    q = rn32(rn32(x * inv + MAGIC) - MAGIC)
    return x - q * m, q


def test_moduli_are_pairwise_coprime_and_their_residues_exact_in_bf16():
    assert len(MODULI) == 16 and max(MODULI) <= 256
    for i, a in enumerate(MODULI):
        for b in MODULI[i + 1:]:
            assert gcd(a, b) == 1
    # symmetric residues lie in [-128, 128]: integers of at most 8 significant bits, which the
    # 8-bit significand of bf16 holds exactly (checked by rounding float32 to bf16)
    r = np.arange(-128, 129, dtype=np.float32)
    bits = r.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    assert np.array_equal(rounded.astype(np.uint32).view(np.float32), r)


@pytest.mark.parametrize("Kp", [64, 1024, 4096, 16384])
def test_plan_keeps_products_below_half_the_modulus(Kp):
    n, p, M = plan(Kp)
    assert p >= 54 and n <= 16
    assert 2 * Kp * 2 ** (2 * p) <= M  # |X| <= Kp (2^p - 1)^2 < M / 2
    if Kp == 16384:
        assert (n, p) == (16, 55)


def test_plan_runs_out_beyond_the_moduli():
    # the product of the 16 moduli is near 2^125.4: no p >= 54 for K' = 2^17
    assert plan(1 << 17) is None
    assert plan(1 << 15) is not None


def test_chunk_sums_are_exact_in_fp32():
    assert CHUNK_BLOCKS * BK * 128 * 128 == 2 ** 24
    rng = np.random.default_rng(3)
    L = CHUNK_BLOCKS * BK
    a = rng.integers(-128, 129, L)
    b = rng.integers(-128, 129, L)
    a[:64] = 128
    b[:64] = 128  # saturated run at the start of the chunk
    exact = int(np.dot(a, b))
    acc = np.float32(0.0)
    for x, y in zip(a.astype(np.float32), b.astype(np.float32)):
        acc = np.float32(acc + np.float32(x * y))
    assert int(acc) == exact
    full = np.full(L, 128)
    assert int(np.dot(full, full)) == 2 ** 24  # the largest chunk sum, still an FP32 integer


@pytest.mark.parametrize("m", MODULI)
def test_fold_is_a_small_congruent_integer(m):
    rng = np.random.default_rng(m)
    xs = [0, 1, -1, 2 ** 24, -(2 ** 24), m // 2, -(m // 2), (m + 1) // 2]
    xs += [int(v) for v in rng.integers(-(2 ** 24), 2 ** 24 + 1, 200)]
    xs += [k * m + m // 2 for k in rng.integers(-(2 ** 24) // m, 2 ** 24 // m, 50)]
    for x in xs:
        r, q = fold32(x, m)
        assert q.denominator == 1 and r.denominator == 1
        assert (x - r) % m == 0
        assert abs(r) <= m // 2 + 2  # q may miss round(x / m) by one next to a half
    # folds of one product accumulate over at most 64 chunks (K' = 65536) far below 2^24
    assert 64 * (256 // 2 + 2) < 2 ** 24


def _weights(n):
    M = prod(MODULI[:n])
    N = [M // m for m in MODULI[:n]]
    y = [pow(Nl % m, -1, m) for Nl, m in zip(N, MODULI[:n])]
    return M, N, y


def test_crt_reconstruction_is_exact():
    Kp = 1024
    n, p, M = plan(Kp)
    Mm, N, y = _weights(n)
    assert Mm == M
    rng = np.random.default_rng(11)
    top = 2 ** p - 1
    rows, cols = 3, 3
    A = [[int(v) for v in rng.integers(-top, top + 1, Kp)] for _ in range(rows)]
    B = [[int(v) for v in rng.integers(-top, top + 1, Kp)] for _ in range(cols)]
    A[0] = [top] * Kp
    B[0] = [top] * Kp  # X = Kp (2^p - 1)^2, the largest product
    B[1] = [-top] * Kp
    for a in A:
        for b in B:
            X = sum(u * v for u, v in zip(a, b))
            t = []
            for l in range(n):
                m = MODULI[l]
                ra = [sym(u, m) for u in a]
                rb = [sym(v, m) for v in b]
                xm = sum(u * v for u, v in zip(ra, rb)) % m  # the tensor product of residues
                t.append(xm * y[l] % m)  # the stored weighted residue
            S = sum(tl * Nl for tl, Nl in zip(t, N))
            Xr = S % M
            if Xr > M // 2:
                Xr -= M
            assert Xr == X


def test_quotient_estimate_from_the_top_limbs_is_within_one():
    n, p, M = plan(1024)
    _, N, _ = _weights(n)
    limbs = lambda v: [(v >> (32 * t)) & 0xFFFFFFFF for t in range(5)]
    top = max(t for t, w in enumerate(limbs(M)) if w)
    b = max(0, top - 1)
    inv_mf = rn32(Fraction(2 ** (32 * b), M))
    rng = np.random.default_rng(5)
    cases = [[m - 1 for m in MODULI[:n]], [0] * n]
    cases += [[int(rng.integers(0, m)) for m in MODULI[:n]] for _ in range(300)]
    for t in cases:
        S = sum(tl * Nl for tl, Nl in zip(t, N))  # S < n M
        s = limbs(S)
        a2, a1, a0 = s[b + 2], s[b + 1], s[b]
        sf = rn32(rn32(a2) * 2 ** 64 + rn32(rn32(a1) * 2 ** 32 + rn32(a0)))
        q = int(rn32(sf * inv_mf))  # truncation toward zero of a non-negative value
        assert abs(q - S // M) <= 1
