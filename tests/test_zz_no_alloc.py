"""gks_gemm_split_noalloc (split product on the library's fixed device scratch) against the
allocating split product of gks_gemm, on two calls in a row, and its size limit."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09058_gb300 import gks
    return gks.Context(0)


def _bound(A, B, K, S=9):
    """Splitting error (digits below 2^{-6S} of the row and column scales) plus the FP64
    rounding of K accumulated terms, twice over for the two products compared."""
    aA, aB = np.abs(A), np.abs(B)
    rowmax, colmax = aA.max(axis=1, keepdims=True), aB.max(axis=0, keepdims=True)
    split = (S + 2) * K * 2.0 ** (-6 * S) * (2 * rowmax) * (2 * colmax)
    return 2.0 * (split + 2 * K * U * (aA @ aB))


def _case(M, N, K, cplx, ops, seed):
    rng = np.random.default_rng(seed)

    def rnd(r, c):
        x = rng.standard_normal((r, c))
        return x + 1j * rng.standard_normal((r, c)) if cplx else x
    A = rnd(*((M, K) if ops[0] == "N" else (K, M)))
    B = rnd(*((K, N) if ops[1] == "N" else (N, K)))
    C0 = rnd(M, N)
    return A, B, C0


def _op(X, op):
    return X if op == "N" else (X.T if op == "T" else X.conj().T)


def test_noalloc_matches_split_gemm_two_calls(ctx):
    dt = {False: torch.float64, True: torch.complex128}
    # two different products back to back on the shared scratch: real, then complex
    cases = [(300, 200, 260, False, ("N", "T"), 1), (130, 90, 150, True, ("C", "N"), 2)]
    for M, N, K, cplx, ops, seed in cases:
        A, B, C0 = _case(M, N, K, cplx, ops, seed)
        Ad = torch.as_tensor(A, dtype=dt[cplx]).cuda()
        Bd = torch.as_tensor(B, dtype=dt[cplx]).cuda()
        ref = ctx.gemm(Ad, Bd, torch.as_tensor(C0, dtype=dt[cplx]).cuda(), ops[0], ops[1], 0.7, -0.3,
                       mode="split").cpu().numpy()
        got = ctx.gemm_split_noalloc(Ad, Bd, torch.as_tensor(C0, dtype=dt[cplx]).cuda(), ops[0], ops[1],
                                     0.7, -0.3).cpu().numpy()
        tol = 0.7 * _bound(_op(A, ops[0]), _op(B, ops[1]), K)
        assert np.all(np.abs(got - ref) <= tol)
        exact = 0.7 * (_op(A, ops[0]) @ _op(B, ops[1])) - 0.3 * C0
        assert np.all(np.abs(got - exact) <= tol + 2 * U * np.abs(0.3 * C0))


def test_noalloc_repeated_call_same_result(ctx):
    A, B, _ = _case(256, 256, 256, False, ("N", "N"), 3)
    Ad, Bd = torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda()
    first = ctx.gemm_split_noalloc(Ad, Bd, torch.zeros(256, 256, dtype=torch.float64, device="cuda")).cpu().numpy()
    second = ctx.gemm_split_noalloc(Ad, Bd, torch.zeros(256, 256, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = ctx.gemm(Ad, Bd, torch.zeros(256, 256, dtype=torch.float64, device="cuda"), mode="split").cpu().numpy()
    tol = _bound(A, B, 256)
    assert np.all(np.abs(first - ref) <= tol)
    assert np.all(np.abs(second - ref) <= tol)


def test_noalloc_rejects_products_beyond_the_scratch(ctx):
    from paper_2606_09058_gb300 import gks
    A = torch.zeros(2048, 2048, dtype=torch.float64, device="cuda")
    C = torch.zeros(2048, 2048, dtype=torch.float64, device="cuda")
    with pytest.raises(gks.GKSError, match="fixed scratch holds"):
        ctx.gemm_split_noalloc(A, A, C)
    # the context stays usable after the rejection
    B = torch.eye(64, dtype=torch.float64, device="cuda")
    out = ctx.gemm_split_noalloc(B, B, torch.zeros(64, 64, dtype=torch.float64, device="cuda"))
    assert torch.equal(out, B)


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_empty_inner_dimension(ctx, cplx):
    """K = 0: no digits to multiply, C = beta C, on the fixed scratch as on the allocating
    path (the scratch takes one zero block of digits)."""
    dt = torch.complex128 if cplx else torch.float64
    A = torch.zeros(64, 0, dtype=dt, device="cuda")
    B = torch.zeros(0, 64, dtype=dt, device="cuda")
    C0 = torch.randn(64, 64, dtype=dt, device="cuda")
    got = ctx.gemm_split_noalloc(A, B, C0.clone(), alpha=0.7, beta=-0.5)
    ref = ctx.gemm(A, B, C0.clone(), alpha=0.7, beta=-0.5, mode="split")
    assert torch.equal(got, ref)
    assert torch.equal(got, -0.5 * C0)
