"""The number format of the one-stage matrix-vector step's digit form, restated in numpy
(no GPU): symmetric power-of-two equilibration A = D Ã D (d_i = ceil(g_i / 2) from the row
maxima), 7 balanced base-256 digits of round(2^54 x) per real part, digit pairs s + t <= 7
summed exactly in integers and weighted by 2^{d_i + fu - 12 - 8L}.  On the reduced Si pencils
(Cholesky and Loewdin routes, whose entries span many decades) its componentwise error,
relative to sum |a_ij| |u_j|, stays within a small multiple of the FP64 unit, and the digits
stay within the signed 8-bit range dp4a takes."""
import math

import numpy as np
import pytest

from paper_2606_09058_gb300 import inputs as I

U64 = 2.0 ** -53


def _bscale(x):
    """e with |x| < 2^e (0 for 0)."""
    _, e = np.frexp(np.abs(x))
    return np.where(x == 0, 0, e).astype(np.int64)


def _digits(x, e):
    """Balanced base-256 digits of round(|x| 2^{54 - e}) with the sign of x, (..., 7)."""
    q = np.floor(np.ldexp(np.abs(x), 55 - e)).astype(np.int64)
    q = (q + 1) >> 1
    v = np.where(x < 0, -q, q)
    d = np.zeros(x.shape + (7,), np.int64)
    for s in range(6, 0, -1):
        t = v & 255
        t = np.where(t >= 128, t - 256, t)
        d[..., s] = t
        v = (v - t) >> 8
    d[..., 0] = v
    return d


def _digit_matvec(A, u):
    g = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=1)
    d = (_bscale(g) + 1) >> 1
    ea = d[:, None] + d[None, :]
    DR, DI = _digits(A.real, ea), _digits(A.imag, ea)
    fu = int((_bscale(np.maximum(np.abs(u.real), np.abs(u.imag))) + d).max())
    UR, UI = _digits(u.real, fu - d), _digits(u.imag, fu - d)
    for X in (DR, DI, UR, UI):
        assert X.min() >= -128 and X.max() <= 127
    p = np.zeros(A.shape[0], complex)
    for r in range(A.shape[0]):
        E = int(d[r]) + fu - 12
        pre = pim = 0.0
        for L in range(7, -1, -1):
            s0 = s1 = s2 = s3 = 0
            for s in range(7):
                t = L - s
                if 0 <= t <= 6:
                    s0 += int(DR[r, :, s] @ UR[:, t])
                    s1 += int(DI[r, :, s] @ UI[:, t])
                    s2 += int(DR[r, :, s] @ UI[:, t])
                    s3 += int(DI[r, :, s] @ UR[:, t])
            pre += math.ldexp(s0 - s1, E - 8 * L)
            pim += math.ldexp(s2 + s3, E - 8 * L)
        p[r] = pre + 1j * pim
    return p


@pytest.mark.parametrize("route", ["cholesky", "lowdin"])
def test_digit_matvec_componentwise_error(route):
    p = I.periodic((1, 1, 1), 1, 0.01)
    H, S = p.H[0].numpy(), p.S[0].numpy()
    if route == "cholesky":
        Li = np.linalg.inv(np.linalg.cholesky(S))
        A = Li @ H @ Li.conj().T
    else:
        s, U = np.linalg.eigh(S)
        V = U / np.sqrt(s)
        A = V.conj().T @ H @ V
    A = 0.5 * (A + A.conj().T)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    u /= np.abs(u).max()
    exact = A.astype(np.clongdouble) @ u.astype(np.clongdouble)
    comp = np.abs(A) @ np.abs(u)
    err = (np.abs(_digit_matvec(A, u) - exact).astype(float) / comp).max()
    assert err <= 16 * U64, err


def test_digits_are_exact_on_integers_and_round_halves_up():
    x = np.array([0.5, -0.25, 1.0 - 2.0 ** -53, 3.0 / 7.0])
    d = _digits(x, np.zeros(4, np.int64))
    val = (d * 2.0 ** (-6 - 8 * np.arange(7))).sum(axis=1)
    assert np.all(np.abs(val - x) <= 2.0 ** -55)
    assert d.min() >= -128 and d.max() <= 127
