"""The split-bf16 FP64 product (gks_gemm mode 2) in both forms, residues (Chinese
remainder) and digit pairs, against numpy's FP64 product and the FP64-pipe kernel, within
the error bound of the splitting: 54 bits relative to each row's and column's largest entry
(so the error scales with K max|a_i.| max|b_.j| rather than with sum |a_ik||b_kj|), plus
the FP64 rounding of K accumulated terms.  Exactness checks drive the FP32 chunk sums of
either form to their 2^24 limit."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09058_gb300 import gks
    return {"residues": gks.Context(0), "digits": gks.Context(0, split="digits")}


@pytest.fixture(scope="module")
def ctx(ctxs):
    return ctxs["residues"]


MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]


def residue_bits(Kp, bits=54):
    """p of the residue form for padded inner length Kp: the fewest moduli whose product M
    has 2 Kp 2^{2p} <= M with p >= bits, p = floor(log2(M // (2 Kp)) / 2) capped at 62."""
    M = 1
    for m in MODULI:
        M *= m
        p = min((M // (2 * Kp)).bit_length() - 1, 124) // 2
        if p >= bits:
            return min(p, 62)
    raise ValueError("no plan")


def _op(X, op):
    return X if op == "N" else (X.T if op == "T" else X.conj().T)


def _bound(A, B, K, S=9):
    """FP64 rounding of the K-term sum plus the splitting error: every digit product and
    the remainders are below 2^{-6S} of the row scale 2^{e_i} <= 2 max_k |a_ik| times the
    column scale (the S + 2 levels at and beyond the truncation, both remainders)."""
    aA, aB = np.abs(A), np.abs(B)
    rowmax, colmax = aA.max(axis=1, keepdims=True), aB.max(axis=0, keepdims=True)
    split = (S + 2) * K * 2.0 ** (-6 * S) * (2 * rowmax) * (2 * colmax)
    return 2.0 * (split + 2 * K * U * (aA @ aB))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("ops", [("N", "N"), ("N", "C"), ("C", "N"), ("T", "T")])
@pytest.mark.parametrize("shape", [(200, 150, 300), (129, 257, 64), (64, 70, 5000), (1, 33, 7)])
@pytest.mark.parametrize("scaling", ["plain", "ill"])
@pytest.mark.parametrize("form", ["residues", "digits"])
def test_split_gemm_accuracy(ctxs, cplx, ops, shape, scaling, form):
    ctx = ctxs[form]
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N + K + cplx)
    def rnd(r, c):
        x = rng.standard_normal((r, c))
        if cplx:
            x = x + 1j * rng.standard_normal((r, c))
        return x
    A = rnd(*((M, K) if ops[0] == "N" else (K, M)))
    B = rnd(*((K, N) if ops[1] == "N" else (N, K)))
    if scaling == "ill":   # rows and columns scaled over 16 decades, entries over 6 decades
        A = A * 10.0 ** rng.uniform(-8, 8, (A.shape[0], 1)) * 10.0 ** rng.uniform(-3, 3, A.shape)
        B = B * 10.0 ** rng.uniform(-8, 8, (1, B.shape[1])) * 10.0 ** rng.uniform(-3, 3, B.shape)
    C0 = rnd(M, N)
    opA, opB = _op(A, ops[0]), _op(B, ops[1])
    ref = 0.7 * (opA @ opB) - 0.3 * C0
    dt = torch.complex128 if cplx else torch.float64
    Ad = torch.as_tensor(A, dtype=dt).cuda()
    Bd = torch.as_tensor(B, dtype=dt).cuda()
    Cs = torch.as_tensor(C0, dtype=dt).cuda()
    Cf = Cs.clone()
    ctx.gemm(Ad, Bd, Cs, ops[0], ops[1], 0.7, -0.3, "split")
    ctx.gemm(Ad, Bd, Cf, ops[0], ops[1], 0.7, -0.3, "fp64")
    bound = 0.7 * _bound(opA, opB, K) + 0.3 * U * np.abs(C0) * 4
    es = np.abs(Cs.cpu().numpy() - ref)
    ef = np.abs(Cf.cpu().numpy() - ref)
    assert np.all(es <= bound), (es / bound).max()
    assert np.all(ef <= bound), (ef / bound).max()


@pytest.mark.parametrize("form", ["residues", "digits"])
def test_split_gemm_is_exact_on_small_integers(ctxs, form):
    """Integer operands below 2^6 are single digits, and integers are exact residues: the
    product is exact."""
    ctx = ctxs[form]
    rng = np.random.default_rng(0)
    A = rng.integers(-63, 64, (300, 700)).astype(float)
    B = rng.integers(-63, 64, (700, 250)).astype(float)
    C = torch.zeros(300, 250, dtype=torch.float64, device="cuda")
    ctx.gemm(torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda(), C, mode="split")
    assert np.array_equal(C.cpu().numpy(), A @ B)


@pytest.mark.parametrize("K", [4096, 4160, 9000])
@pytest.mark.parametrize("signs", ["positive", "mixed"])
def test_split_gemm_saturated_digits(ctxs, K, signs):
    """Entries 1 - 2^-52 have (nearly) all 54 digit bits set, so every digit product is
    63^2 and the exact FP32 partial sums reach their 2^24 limit.  A single lost bit in the
    leading level would be an error of 2^-12 per element, far above the splitting bound
    (which the dropped pairs s + t > S + 1 nearly reach here)."""
    ctx = ctxs["digits"]
    x = 1.0 - 2.0 ** -52
    rng = np.random.default_rng(K)
    A = np.full((130, K), x)
    B = np.full((K, 140), x)
    if signs == "mixed":
        A *= rng.choice([-1.0, 1.0], A.shape)
        B *= rng.choice([-1.0, 1.0], B.shape)
    C = torch.zeros(130, 140, dtype=torch.float64, device="cuda")
    ctx.gemm(torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda(), C, mode="split")
    # exact: (A B)_ij = x^2 * (integer sign sum), x^2 = 1 - 2^-51 + 2^-104
    ssum = np.sign(A) @ np.sign(B)
    ref = ssum * x * x
    assert np.all(np.abs(C.cpu().numpy() - ref) <= _bound(A, B, K))


@pytest.mark.parametrize("form", ["residues", "digits"])
def test_solve_with_split_products_matches_oracle(ctx, form):
    """Full path with every product forced through split products, on the Si cluster."""
    from oracle import oracle as O
    from paper_2606_09058_gb300 import gks, inputs as I
    c2 = gks.Context(0, gemm="split", split=form)
    for p in (I.collinear_gamma((2, 1, 1), 0, 0.01), I.periodic((1, 1, 1), 1, 0.01)):
        sol = c2.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, kweights=torch.as_tensor(p.kweights).cuda())
        ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, kweights=p.kweights)
        for k in range(p.nk):
            H, S = p.H[k].numpy(), p.S[k].numpy()
            beta = O.eig_condition(H, S, ref.eps[k], ref.C[k])
            assert np.all(np.abs(sol.eps.cpu().numpy()[k] - ref.eps[k]) <= np.maximum(1e-10, 8 * beta))
            C = sol.C.cpu().numpy()[k]
            cn = np.linalg.norm(C, axis=0)
            R = H @ C - (S @ C) * sol.eps.cpu().numpy()[k]
            bwd = (np.linalg.norm(R, axis=0) / ((np.linalg.norm(H, 2) + np.abs(ref.eps[k]) * np.linalg.norm(S, 2)) * cn)).max()
            assert bwd <= 1e-12 * np.sqrt(H.shape[0])
            d = np.abs(S @ (sol.rho.cpu().numpy()[k] - ref.rho[k]) @ S).max()
            assert d <= 1e-9 * max(1.0, beta.max() / 1e-10)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("mode", ["split", "fp64", "digits"])
def test_gemm_empty_inner_dimension(ctxs, cplx, mode):
    """K = 0 gives C = beta C on every product path."""
    ctx = ctxs["digits" if mode == "digits" else "residues"]
    mode = "split" if mode == "digits" else mode
    dt = torch.complex128 if cplx else torch.float64
    A = torch.zeros(300, 0, dtype=dt, device="cuda")
    B = torch.zeros(0, 200, dtype=dt, device="cuda")
    C0 = torch.randn(300, 200, dtype=dt, device="cuda")
    out = ctx.gemm(A, B, C0.clone(), alpha=2.0, beta=0.25, mode=mode)
    assert torch.equal(out, 0.25 * C0)


@pytest.mark.parametrize("K", [1024, 4096, 5000])
@pytest.mark.parametrize("signs", ["positive", "mixed"])
@pytest.mark.parametrize("cplx", [False, True])
def test_split_gemm_saturated_residues(ctx, K, signs, cplx):
    """Entries a = 1/2 + 2^{7-p} (p the residue form's bits for this K) truncate to the
    integer 2^{p-1} + 128, whose residue modulo 256 is +128: every product of that plane is
    2^14 and a 1024-long chunk sums to exactly 2^24, the limit of the FP32 accumulator.
    The integer product is rebuilt exactly, so C is the correctly rounded A B (bit for bit).
    Complex: the imaginary parts are the same value (embedded inner length 2K)."""
    Ke = 2 * K if cplx else K
    p = residue_bits(-(-Ke // 64) * 64)
    q = 2 ** (p - 1) + 128
    a = q / 2.0 ** p
    assert a * 2.0 ** p == q and 0.5 <= a < 1.0
    rng = np.random.default_rng(K + 7 * cplx)
    sa = np.ones((130, K)) if signs == "positive" else rng.choice([-1.0, 1.0], (130, K))
    sb = np.ones((K, 140)) if signs == "positive" else rng.choice([-1.0, 1.0], (K, 140))
    A, B = a * sa, a * sb
    if cplx:
        A, B = A + 1j * a * sa, B + 1j * a * sb
    dt = torch.complex128 if cplx else torch.float64
    C = torch.zeros(130, 140, dtype=dt, device="cuda")
    ctx.gemm(torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda(), C, mode="split")
    # exact: integer sign sums times q^2 2^{-2p}; complex: (1 + i)^2 = 2i
    ssum = (sa @ sb).astype(np.int64)
    ref = np.array([[float((int(v) * q * q) / 2 ** (2 * p)) for v in row] for row in ssum])
    got = C.cpu().numpy()
    if cplx:
        assert np.array_equal(got.real, np.zeros_like(ref))
        assert np.array_equal(got.imag, np.array([[float((2 * int(v) * q * q) / 2 ** (2 * p)) for v in row]
                                                   for row in ssum]))
    else:
        assert np.array_equal(got, ref)
