"""Two-stage tridiagonalization through the C ABI against the oracle's stage references:
dense -> band (oracle.band_reduce_blocked: the same reflector convention, so the band
matrix and Q1 match entry by entry), band -> tridiagonal by bulge chasing (oracle.bulge_chase:
the tridiagonal and Q2 entry by entry, the last off-diagonal up to its phase, which the GPU
path makes real with one more one-element reflector), Q2 applied to a block of columns,
reconstruction and unitarity, the full two-stage solve (all eigenvectors and the lowest
n_ev) on the parity gates, and the chase's bounded waits."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2606_09058_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09058_gb300 import gks as g
    return g


def _herm(n, seed, cplx):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    if cplx:
        A = A + 1j * rng.standard_normal((n, n))
    return 0.5 * (A + A.conj().T)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(12, 3), (37, 4), (130, 8), (301, 32)])
def test_he2hb_matches_oracle(gks, cplx, n, b):
    A = _herm(n, 10 * n + b, cplx)
    ctx = gks.Context(0)
    Bd, Qd = ctx.he2hb(torch.as_tensor(np.tril(A)).cuda(), b, want_q=True)
    B, Q = Bd.cpu().numpy()[0], Qd.cpu().numpy()[0]
    Bo, Qo = O.band_reduce_blocked(A, b)
    scale = np.abs(A).max() * n
    i, j = np.indices((n, n))
    assert np.all(B[np.abs(i - j) > b] == 0)
    assert np.abs(B - Bo).max() <= 1e-13 * scale, np.abs(B - Bo).max()
    assert np.abs(Q - Qo).max() <= 1e-13 * n
    assert np.abs(Q @ B @ Q.conj().T - A).max() <= 1e-13 * scale
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 1e-13 * n


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(12, 3), (40, 4), (97, 8), (260, 32)])
def test_hb2st_matches_oracle(gks, cplx, n, b):
    A = _herm(n, 7 * n + b, cplx)
    Bo, _ = O.band_reduce(A, b)
    Bo = 0.5 * (Bo + Bo.conj().T)
    i, j = np.indices((n, n))
    Bo[np.abs(i - j) > b] = 0.0
    refl = []
    To, Q2o = O.bulge_chase(Bo, b, refl)
    ctx = gks.Context(0)
    X = torch.eye(n, dtype=torch.complex128 if cplx else torch.float64, device="cuda")[None].contiguous()
    d, e = ctx.hb2st(torch.as_tensor(Bo).cuda(), b, X)
    d, e, Q2 = d.cpu().numpy()[0], e.cpu().numpy()[0], X.cpu().numpy()[0]
    scale = np.abs(Bo).max() * n
    assert np.abs(d - np.real(np.diag(To))).max() <= 1e-13 * scale
    sub = np.diag(To, -1)
    assert np.abs(e[:n - 2] - np.real(sub[:n - 2])).max() <= 1e-13 * scale
    assert np.abs(np.imag(sub[:n - 2])).max() <= 1e-13 * scale
    assert abs(abs(e[n - 2]) - abs(sub[n - 2])) <= 1e-13 * scale
    # Q2: all columns but the last as the oracle's; the last up to a unit phase
    assert np.abs(Q2[:, :n - 1] - Q2o[:, :n - 1]).max() <= 1e-12 * n
    ph = np.vdot(Q2o[:, n - 1], Q2[:, n - 1])
    assert abs(abs(ph) - 1.0) <= 1e-12 and np.abs(Q2[:, n - 1] - ph * Q2o[:, n - 1]).max() <= 1e-12 * n
    T = np.diag(d) + np.diag(e[:n - 1], -1) + np.diag(e[:n - 1], 1)
    assert np.abs(Q2 @ T @ Q2.conj().T - Bo).max() <= 1e-13 * scale
    # the grouped application of the oracle's reflectors to a block of columns
    rng = np.random.default_rng(n)
    nc = min(17, n)
    Y = rng.standard_normal((n, nc)) + (1j * rng.standard_normal((n, nc)) if cplx else 0)
    Yd = torch.as_tensor(Y).cuda()[None].contiguous()
    ctx.hb2st(torch.as_tensor(Bo).cuda(), b, Yd)
    # the GPU's Q2 is the oracle's times diag(1, .., 1, ph) (its last one-element reflector)
    Yph = np.array(Y, dtype=np.result_type(Y, ph))
    Yph[n - 1] *= ph
    Yo = O.apply_q2_grouped(refl, Yph, b)
    got = Yd.cpu().numpy()[0]
    assert np.abs(got - Yo).max() <= 1e-12 * n * np.abs(Y).max()


def _scaled(H, S, eps, C):
    nh, ns = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    cn = np.linalg.norm(C, axis=0)
    G = C.conj().T @ S @ C - np.eye(C.shape[1])
    orth = np.abs(G / np.outer(cn, cn) / ns).max()
    R = H @ C - (S @ C) * eps
    bwd = (np.linalg.norm(R, axis=0) / ((nh + np.abs(eps) * ns) * cn)).max()
    return orth, bwd


def _check(sol, p, spin="collinear", n_ev=0):
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, spin, p.kweights)
    eps, C, rho = sol.eps.cpu().numpy(), sol.C.cpu().numpy(), sol.rho.cpu().numpy()
    nk, M = eps.shape
    for k in range(nk):
        Sk = O.spinor_overlap(p.S[k].numpy()) if spin == "noncollinear" else p.S[k].numpy()
        Hk = p.H[k].numpy()
        beta = O.eig_condition(Hk, Sk, ref.eps[k], ref.C[k])
        assert np.all(np.abs(eps[k] - ref.eps[k]) <= np.maximum(1e-10, 8 * beta)), np.abs(eps[k] - ref.eps[k]).max()
        ncol = C.shape[-1]
        orth, bwd = _scaled(Hk, Sk, eps[k][:ncol], C[k])
        assert orth <= 1e-12 * math.sqrt(M) and bwd <= 1e-12 * math.sqrt(M), (orth, bwd)
        d = np.abs(Sk @ (rho[k] - ref.rho[k]) @ Sk).max()
        assert d <= 1e-9 * max(1.0, beta.max() / 1e-10), d
    assert abs(sol.mu.item() - ref.mu) <= 1e-3 * p.kT


@pytest.mark.parametrize("band", [8, 32])
def test_two_stage_solve_si_and_kbatch(gks, band):
    ctx = gks.Context(0, tridiag="two_stage", band=band)
    for p in (I.collinear_gamma((2, 1, 1), 0, 0.01), I.periodic((1, 1, 1), 1, 0.01)):
        sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, kweights=torch.as_tensor(p.kweights).cuda())
        _check(sol, p)


@pytest.mark.parametrize("cplx,m", [(False, 389), (True, 301), (False, 1100)])
def test_two_stage_solve_random_pencil(gks, cplx, m):
    H, S = I.random_pencil(m, 1300 + m, cplx, cond=1e2)
    ctx = gks.Context(0, tridiag="two_stage")
    sol = ctx.solve(torch.as_tensor(H)[None].cuda(), torch.as_tensor(S)[None].cuda(), 0.1, 0.6 * m)
    ref = O.solve(H[None], S[None], 0.1, 0.6 * m)
    eps, C = sol.eps[0].cpu().numpy(), sol.C[0].cpu().numpy()
    assert np.abs(eps - ref.eps[0]).max() <= 1e-10 * max(1.0, np.abs(ref.eps[0]).max())
    orth, bwd = _scaled(H, S, eps, C)
    assert orth <= 1e-12 * math.sqrt(m) and bwd <= 1e-12 * math.sqrt(m), (orth, bwd)
    assert np.abs(S @ (sol.rho[0].cpu().numpy() - ref.rho[0]) @ S).max() <= 1e-9


def test_two_stage_noncollinear_and_partial_spectrum(gks):
    p = I.noncollinear((1, 1, 1), 2, 0.01)
    ctx = gks.Context(0, tridiag="two_stage")
    _check(ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, "noncollinear"), p, "noncollinear")
    q = I.periodic((1, 1, 1), 1, 0.01)
    ref = O.solve(q.H.numpy(), q.S.numpy(), q.kT, q.n_elec, kweights=q.kweights)
    cp = gks.Context(0, tridiag="two_stage", n_ev=int(ref.n_rho.max()) + 5)
    _check(cp.solve(q.H.cuda(), q.S.cuda(), q.kT, q.n_elec, kweights=torch.as_tensor(q.kweights).cuda()), q)


def test_bulge_chase_wait_expires(gks):
    """A wait limit of one cycle: the second sweep's first wait on the first sweep's progress
    expires, every worker stops (no hang), gks_sync reports GKS_ETIMEOUT; a context with the
    default limit then reduces the same band correctly."""
    n, b = 200, 8
    A = _herm(n, 5, True)
    Bo, _ = O.band_reduce(A, b)
    Bo = 0.5 * (Bo + Bo.conj().T)
    i, j = np.indices((n, n))
    Bo[np.abs(i - j) > b] = 0.0
    short = gks.Context(0, wait_limit=1)
    with pytest.raises(gks.GKSError) as ei:
        short.hb2st(torch.as_tensor(Bo).cuda(), b)
    assert ei.value.code == gks.GKS_ETIMEOUT
    d, e = gks.Context(0).hb2st(torch.as_tensor(Bo).cuda(), b)
    T = np.diag(d.cpu().numpy()[0]) + np.diag(e.cpu().numpy()[0][:n - 1], -1) + np.diag(e.cpu().numpy()[0][:n - 1], 1)
    assert np.abs(np.linalg.eigvalsh(T) - np.linalg.eigvalsh(A)).max() <= 1e-12 * n
