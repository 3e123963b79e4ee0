"""Parity of the CUDA path (through the C ABI) with the CPU oracle, stage by stage and
end to end, on seeded inputs that span several 64-wide panels and a ragged tail.

Tolerances: closed-form and well-conditioned pencils use the raw gates (|d eps| <= 1e-10
relative to the spectrum scale, orthonormality and backward error <= 1e-12 sqrt(M));
the Si Gaussian basis (kappa(S) ~ 1e10) uses the condition-scaled gates: per eigenvalue
|d eps_i| <= max(1e-10, 8 beta_i) with beta_i = u (||H|| + |eps_i| ||S||) ||c_i||^2, and
the density matrix compared S-covariantly, ||S (rho - rho_ref) S||_max."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2606_09058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09058_gb300 import gks
    return gks.Context(0)


def _cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _scaled(H, S, eps, C):
    nh, ns = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    cn = np.linalg.norm(C, axis=0)
    G = C.conj().T @ S @ C - np.eye(C.shape[1])
    orth = np.abs(G / np.outer(cn, cn) / ns).max()
    R = H @ C - (S @ C) * eps
    bwd = (np.linalg.norm(R, axis=0) / ((nh + np.abs(eps) * ns) * cn)).max()
    return orth, bwd


# ------------------------------------------------------------------ stages

@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m", [1, 5, 63, 64, 65, 130, 333])
def test_potrf_matches_oracle(ctx, cplx, m):
    _, S = I.random_pencil(m, 100 + m, cplx, cond=1e6)
    L = ctx.potrf(_cuda(S)).cpu().numpy()[0]
    ref = O.cholesky(S)
    assert np.abs(np.tril(L) - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


def test_potrf_reports_failing_column(ctx):
    from paper_2606_09058_gb300 import gks
    S = np.eye(150)
    S[97, 97] = -1.0
    with pytest.raises(gks.GKSError) as ei:
        ctx.potrf(_cuda(S))
    assert ei.value.code == gks.GKS_ENOTSPD and "column 97" in str(ei.value)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m", [1, 7, 64, 100, 200])
def test_reduce_matches_oracle(ctx, cplx, m):
    H, S = I.random_pencil(m, 200 + m, cplx, cond=1e3)
    Hd, _ = ctx.reduce(_cuda(H), _cuda(S))
    Hp = np.tril(Hd.cpu().numpy()[0])
    ref = O.reduce_standard(O.cholesky(S), H)
    assert np.abs(Hp - np.tril(ref)).max() <= 1e-12 * m * max(1.0, np.abs(ref).max())


def _tridiag_case(kind, m, rng):
    if kind == "random":
        return rng.standard_normal(m), rng.standard_normal(m)
    if kind == "clustered":
        return 1.0 + 1e-12 * rng.standard_normal(m), 1e-9 * rng.standard_normal(m)
    if kind == "wilkinson":
        h = (m - 1) / 2.0
        return np.abs(np.arange(m) - h), np.ones(m)
    if kind == "split":
        d, e = rng.standard_normal(m), rng.standard_normal(m)
        e[:: max(1, m // 7)] = 0.0
        return d, e
    if kind == "glued":  # repeated blocks: massive deflation of equal poles
        blk = rng.standard_normal(8)
        d = np.tile(blk, m // 8 + 1)[:m]
        e = np.tile(np.r_[np.full(7, 0.5), 1e-14], m // 8 + 1)[:m]
        return d, e
    return np.zeros(m), np.zeros(m)


@pytest.mark.parametrize("kind", ["random", "clustered", "wilkinson", "split", "glued", "zero"])
@pytest.mark.parametrize("m", [1, 2, 3, 31, 32, 33, 64, 100, 257, 1000])
def test_stedc_matches_oracle(ctx, kind, m):
    rng = np.random.default_rng(7 * m + len(kind))
    d, e = _tridiag_case(kind, m, rng)
    e = np.asarray(e, float).copy()
    e[m - 1] = 0.0
    lam, Z = ctx.stedc(_cuda(d), _cuda(e))
    lam, Z = lam.cpu().numpy()[0], Z.cpu().numpy()[0]
    ref, _ = O.tridiagonal_eig(d, e[: m - 1])
    T = np.diag(d) + np.diag(e[: m - 1], 1) + np.diag(e[: m - 1], -1)
    scale = max(1.0, np.abs(T).max())
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(lam - ref).max() <= 1e-13 * math.sqrt(m) * scale * 10
    assert np.abs(Z.T @ Z - np.eye(m)).max() <= 1e-13 * m
    assert np.abs(T @ Z - Z * lam).max() <= 1e-13 * m * scale


# ------------------------------------------------------------------ full path

def _compare(ctx, H, S, kT, n_elec, spin="collinear", kweights=None, raw=False):
    sol = ctx.solve(_cuda(H), _cuda(S), kT, n_elec, spin,
                    None if kweights is None else _cuda(np.asarray(kweights, float)))
    ref = O.solve(H, S, kT, n_elec, spin, kweights)
    eps, C, rho = sol.eps.cpu().numpy(), sol.C.cpu().numpy(), sol.rho.cpu().numpy()
    nk, M = eps.shape
    tr = 0.0
    w = np.full(nk, 1.0 / nk) if kweights is None else np.asarray(kweights)
    bmax = 0.0
    for k in range(nk):
        Sk = O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k]
        beta = O.eig_condition(H[k], Sk, ref.eps[k], ref.C[k])
        bmax = max(bmax, beta.max())
        tol = np.full(M, 1e-10 * max(1.0, np.abs(ref.eps[k]).max())) if raw else np.maximum(1e-10, 8 * beta)
        assert np.all(np.abs(eps[k] - ref.eps[k]) <= tol), f"k={k} max |d eps| {np.abs(eps[k] - ref.eps[k]).max()}"
        orth, bwd = _scaled(H[k], Sk, eps[k], C[k])
        assert orth <= 1e-12 * math.sqrt(M), f"k={k} orthonormality {orth}"
        assert bwd <= 1e-12 * math.sqrt(M), f"k={k} backward error {bwd}"
        drho = np.abs(Sk @ (rho[k] - ref.rho[k]) @ Sk).max()
        assert drho <= 1e-9 * (1.0 if raw else max(1.0, beta.max() / 1e-10)), f"k={k} |S drho S| {drho}"
        assert np.abs(rho[k] - rho[k].conj().T).max() == 0.0
        tr += w[k] * np.trace(rho[k] @ Sk).real
    assert abs(tr - n_elec) <= 1e-9 * n_elec * max(1.0, bmax / 1e-10)
    assert abs(sol.mu.item() - ref.mu) <= max(1e-9, 1e-3 * kT)
    assert abs(sol.e_band.item() - ref.e_band) <= 1e-9 * max(1.0, abs(ref.e_band)) * max(1.0, bmax / 1e-10)
    return sol, ref


@pytest.mark.parametrize("n", [1, 2, 50, 161])
def test_solve_chain_closed_form(ctx, n):
    H, S = I.chain(n, 0.3, -1.0)
    sol, _ = _compare(ctx, H[None], S[None], 0.05, float(n) if n > 1 else 1.0, raw=True)
    ref = 0.3 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    assert np.abs(sol.eps.cpu().numpy()[0] - ref).max() <= 1e-13 * n


def test_solve_twisted_ring_closed_form(ctx):
    n, phi = 64, 2.5
    H, S = I.twisted_ring(n, 0.1, 0.8, phi)
    sol, _ = _compare(ctx, H[None], S[None], 0.05, 40.0, raw=True)
    ref = np.sort(0.1 + 1.6 * np.cos((2 * np.pi * np.arange(n) + phi) / n))
    assert np.abs(sol.eps.cpu().numpy()[0] - ref).max() <= 1e-13 * n


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m", [97, 150])
def test_solve_random_pencil(ctx, cplx, m):
    H, S = I.random_pencil(m, 300 + m, cplx, cond=1e2)
    _compare(ctx, H[None], S[None], 0.1, 0.6 * m, raw=True)


@pytest.mark.parametrize("cplx,m", [(False, 1100), (True, 1030)])
def test_solve_random_pencil_large(ctx, cplx, m):
    """Orders past 1024: the top divide-and-conquer merges and (complex) the density matrix
    run as split products."""
    H, S = I.random_pencil(m, 700 + m, cplx, cond=1e2)
    _compare(ctx, H[None], S[None], 0.1, 0.6 * m, raw=True)


@pytest.mark.parametrize("tiling", [(1, 1, 1), (2, 1, 1)])
def test_solve_si_cluster(ctx, tiling):
    p = I.collinear_gamma(tiling, 0, 0.01)
    _compare(ctx, p.H.numpy(), p.S.numpy(), p.kT, p.n_elec)


def test_solve_gamma64_workload(ctx):
    """64-atom cluster, N = 832 real, kT 0.01, n_elec 256."""
    p = I.workload("gamma64")
    _compare(ctx, p.H.numpy(), p.S.numpy(), p.kT, p.n_elec)


def test_solve_kbatch_shared_mu(ctx):
    """8 Monkhorst-Pack k-points of a one-cell supercell solved as one batch, shared mu."""
    p = I.periodic((1, 1, 1), 1, 0.01)
    sol, ref = _compare(ctx, p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, kweights=p.kweights)
    kf = p.meta["kpoints"]
    eps = sol.eps.cpu().numpy()
    for a in range(p.nk):
        b = int(np.argmin(np.abs(kf + kf[a]).sum(1)))
        beta = O.eig_condition(p.H[a].numpy(), p.S[a].numpy(), ref.eps[a], ref.C[a])
        assert np.all(np.abs(eps[a] - eps[b]) <= np.maximum(1e-10, 16 * beta))


def test_solve_noncollinear(ctx):
    p = I.noncollinear((1, 1, 1), 2, 0.01)
    _compare(ctx, p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, spin="noncollinear")


def test_solve_noncollinear_zero_mixing_doubles(ctx):
    p = I.noncollinear((1, 1, 1), 2, 0.01, delta=0.0, lam=0.0)
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, "noncollinear")
    ec, Cc = O.eigh_generalized(p.meta["H"].numpy(), p.meta["S"].numpy())
    beta = O.eig_condition(p.meta["H"].numpy(), p.meta["S"].numpy(), ec, Cc)
    eps = sol.eps.cpu().numpy()[0]
    tol = np.maximum(1e-10, 16 * beta)
    assert np.all(np.abs(eps[0::2] - ec) <= tol) and np.all(np.abs(eps[1::2] - ec) <= tol)


# ------------------------------------------------------------------ edge cases and errors

def test_solve_rejects_bad_arguments(ctx):
    from paper_2606_09058_gb300 import gks
    H, S = I.chain(10, 0.0, -1.0)
    with pytest.raises(gks.GKSError) as ei:
        ctx.solve(_cuda(H), _cuda(S), 0.0, 10.0)
    assert ei.value.code == gks.GKS_EINVAL
    with pytest.raises(gks.GKSError) as ei:
        ctx.solve(_cuda(H), _cuda(S), 0.01, 20.0)
    assert ei.value.code == gks.GKS_EINVAL


def test_solve_reports_not_positive_definite(ctx):
    from paper_2606_09058_gb300 import gks
    H, S = I.chain(80, 0.0, -1.0)
    S = S.copy()
    S[70, 70] = -2.0
    with pytest.raises(gks.GKSError) as ei:
        ctx.solve(_cuda(H), _cuda(S), 0.01, 10.0)
    assert ei.value.code == gks.GKS_ENOTSPD and "column 70" in str(ei.value)
    # the context stays usable
    H2, S2 = I.chain(80, 0.0, -1.0)
    ctx.solve(_cuda(H2), _cuda(S2), 0.01, 10.0)


# ------------------------------------------------------------------ outer block widths

@pytest.fixture(scope="module", params=[64, 128, 192, 512])
def ctx_block(request, ctx):
    from paper_2606_09058_gb300 import gks
    return gks.Context(0, block=request.param)


@pytest.mark.parametrize("cplx", [False, True])
def test_blocked_potrf_and_reduce_outer_widths(ctx_block, cplx):
    """Two-level Cholesky and reduction with several outer panels and a ragged tail."""
    m = 461
    H, S = I.random_pencil(m, 500 + cplx, cplx, cond=1e3)
    L = ctx_block.potrf(_cuda(S)).cpu().numpy()[0]
    Lr = O.cholesky(S)
    assert np.abs(np.tril(L) - Lr).max() <= 1e-11 * max(1.0, np.abs(Lr).max())
    Hd, _ = ctx_block.reduce(_cuda(H), _cuda(S))
    ref = O.reduce_standard(Lr, H)
    assert np.abs(np.tril(Hd.cpu().numpy()[0]) - np.tril(ref)).max() <= 1e-12 * m * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("cplx", [False, True])
def test_blocked_solve_outer_widths(ctx_block, cplx):
    """Full solve (two-level back-transforms included) for each outer width."""
    m = 389
    H, S = I.random_pencil(m, 600 + cplx, cplx, cond=1e2)
    _compare(ctx_block, H[None], S[None], 0.1, 0.6 * m, raw=True)


# ------------------------------------------------------------------ FP64-pipe-only products

@pytest.mark.parametrize("cplx,m", [(False, 461), (True, 389)])
def test_solve_fp64_products_only(cplx, m):
    """Every product on the FP64 pipe (no split products): the plain FP64 form of the path."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_09058_gb300 import gks
    c64 = gks.Context(0, gemm="fp64", block=128)
    H, S = I.random_pencil(m, 900 + m, cplx, cond=1e2)
    _compare(c64, H[None], S[None], 0.1, 0.6 * m, raw=True)
