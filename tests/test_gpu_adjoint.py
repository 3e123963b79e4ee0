"""Adjoint (gks_adjoint) parity with the oracle adjoint, finite differences of the CUDA
solve, the free-energy identity, and the torch.autograd.Function wrapper."""
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


def _orth(G, L):
    """Gradient in orthonormalized coordinates: for dX = L Gd L^H, dL = Re tr((L^H X L)^H Gd)."""
    return L.conj().T @ G @ L


@pytest.mark.parametrize("case", ["random", "random_complex", "si_cluster", "kbatch", "noncollinear"])
def test_adjoint_matches_oracle(ctx, case):
    rng = np.random.default_rng(5)
    spin, kw = "collinear", None
    if case.startswith("random"):
        H, S = I.random_pencil(70, 9, case.endswith("complex"), 10.0)
        H, S, kT, ne = H[None], S[None], 0.1, 50.0
    elif case == "si_cluster":
        p = I.collinear_gamma((1, 1, 1), 3, 0.02)
        H, S, kT, ne = p.H.numpy(), p.S.numpy(), p.kT, p.n_elec
    elif case == "kbatch":
        p = I.periodic((1, 1, 1), 1, 0.01)
        H, S, kT, ne, kw = p.H.numpy(), p.S.numpy(), 0.05, p.n_elec, p.kweights
    else:
        p = I.noncollinear((1, 1, 1), 2, 0.02)
        H, S, kT, ne, spin = p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, "noncollinear"
    nk, M = H.shape[0], H.shape[1]
    ref = O.solve(H, S, kT, ne, spin, kw)
    rho_t = ref.rho + 0.01 * rng.standard_normal(ref.rho.shape)
    a_eps = 0.1 * rng.standard_normal((nk, M))
    # loss = E_band + tr(D S D S) per k + a.eps, D = rho - rho_t  ->  rho_bar = 2 S D S
    rb_ref = np.stack([2.0 * (O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k])
                       @ (ref.rho[k] - rho_t[k]) @ (O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k])
                       for k in range(nk)])
    Hb_ref, Sb_ref = O.adjoint(ref, kT, spin, kw, rho_bar=rb_ref, eps_bar=a_eps, e_band_bar=1.0)
    kwd = None if kw is None else _cuda(np.asarray(kw, float))
    sol = ctx.solve(_cuda(H), _cuda(S), kT, ne, spin, kwd)
    rho = sol.rho.cpu().numpy()
    rb = np.stack([2.0 * (O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k])
                   @ (rho[k] - rho_t[k]) @ (O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k])
                   for k in range(nk)])
    Hb, Sb = ctx.adjoint(sol, _cuda(S), kT, spin, kwd, rho_bar=_cuda(rb), eps_bar=_cuda(a_eps), e_band_bar=1.0)
    Hb, Sb = Hb.cpu().numpy(), Sb.cpu().numpy()
    # Scale of the FP64 conditioning noise: the same adjoint formulas fed with a second,
    # independent FP64 eigensolver (LAPACK) instead of the oracle's eigenpairs.
    tol_h, tol_s = 1e-6, 1e-6
    if not case.startswith("random"):
        import scipy.linalg as sl
        lap_eps, lap_C = [], []
        for k in range(nk):
            Sk = O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k]
            wv, V = sl.eigh(H[k], Sk)
            lap_eps.append(wv)
            lap_C.append(O.phase_fix(V))
        lap_eps, lap_C = np.stack(lap_eps), np.stack(lap_C)
        gs_ = 1.0 if spin == "noncollinear" else 2.0
        wk = np.full(nk, 1.0 / nk) if kw is None else np.asarray(kw)
        mu_l = O.chemical_potential(lap_eps, wk, gs_, kT, ne)
        occ_l = np.stack([O.fermi((lap_eps[k] - mu_l) / kT) for k in range(nk)])
        rho_l = np.stack([O.density_matrix(lap_C[k], occ_l[k], gs_) for k in range(nk)])
        lap = O.Result(lap_eps, lap_C, mu_l, occ_l, rho_l, 0.0, None)
        rb_l = np.stack([2.0 * (O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k])
                         @ (rho_l[k] - rho_t[k]) @ (O.spinor_overlap(S[k]) if spin == "noncollinear" else S[k])
                         for k in range(nk)])
        Hb_l, Sb_l = O.adjoint(lap, kT, spin, kw, rho_bar=rb_l, eps_bar=a_eps, e_band_bar=1.0)
        sh = ss = 0.0
        for k in range(nk):
            Lc = np.linalg.cholesky(S[k])
            Ls = O.spinor_overlap(Lc) if spin == "noncollinear" else Lc
            r = _orth(Hb_ref[k], Ls)
            sh = max(sh, np.abs(_orth(Hb_l[k], Ls) - r).max() / np.abs(r).max())
            r = _orth(Sb_ref[k], Lc)
            ss = max(ss, np.abs(_orth(Sb_l[k], Lc) - r).max() / np.abs(r).max())
        tol_h, tol_s = max(1e-6, 4.0 * sh), max(1e-6, 4.0 * ss)
    for k in range(nk):
        Lc = np.linalg.cholesky(S[k])
        Ls = O.spinor_overlap(Lc) if spin == "noncollinear" else Lc
        gh, gh_ref = _orth(Hb[k], Ls), _orth(Hb_ref[k], Ls)
        gs, gs_ref = _orth(Sb[k], Lc), _orth(Sb_ref[k], Lc)
        assert np.abs(gh - gh_ref).max() <= tol_h * np.abs(gh_ref).max(), (np.abs(gh - gh_ref).max(), tol_h)
        assert np.abs(gs - gs_ref).max() <= tol_s * np.abs(gs_ref).max(), (np.abs(gs - gs_ref).max(), tol_s)
        assert np.abs(Hb[k] - Hb[k].conj().T).max() == 0.0


def test_adjoint_free_energy_identity(ctx):
    """With explicit eigenvalue weights w g_s f the adjoint returns dF/dH = rho exactly."""
    p = I.collinear_gamma((2, 1, 1), 0, 0.01)
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec)
    eps = sol.eps.cpu().numpy()
    f = O.fermi((eps - sol.mu.item()) / p.kT)
    Hb, _ = ctx.adjoint(sol, p.S.cuda(), p.kT, eps_bar=_cuda(2.0 * f))
    rho = sol.rho.cpu().numpy()[0]
    S = p.S.numpy()[0]
    d = np.abs(S @ (Hb.cpu().numpy()[0] - rho) @ S).max()
    assert d <= 1e-9 * np.abs(S @ rho @ S).max()


def _fd_check(ctx, n, ndir, h, gate, seed):
    """Loss E_band + ||rho - rho_t||_F^2 on a random well-conditioned real pencil of order
    n, kT = 0.02, rho_t the density matrix of a seeded perturbed H (H + 1e-3 S U2 S).
    Directions D = L G L^T (G of unit Frobenius norm), ndir in H and ndir in S; fourth-
    order central differences of the CUDA solve against the CUDA adjoint must agree to
    `gate` relative plus the difference quotient's own noise, 20 sigma/h, with sigma the
    measured rounding noise of the loss, at least one rounding unit of the loss value (the
    plain FP64 oracle itself misses a bare 1e-6 gate at n = 400 on its smallest
    derivatives)."""
    kT = 0.02
    H, S = I.random_pencil(n, seed, False, 10.0)
    ne = 0.6 * n
    rng = np.random.default_rng(seed)
    U2 = rng.uniform(-1.0, 1.0, (n, n))
    U2 = 0.5 * (U2 + U2.T)
    Hd, Sd = _cuda(H[None]), _cuda(S[None])
    rho_t = ctx.solve(_cuda((H + 1e-3 * S @ U2 @ S)[None]), Sd, kT, ne).rho.clone()
    base = ctx.solve(Hd, Sd, kT, ne)

    def loss(Hx, Sx):
        s = ctx.solve(Hx, Sx, kT, ne)
        return float(s.e_band.item() + ((s.rho - rho_t) ** 2).sum().item())

    Hb, Sb = ctx.adjoint(base, Sd, kT, rho_bar=2.0 * (base.rho - rho_t), e_band_bar=1.0)
    Lc = torch.linalg.cholesky(Sd[0])
    # rounding noise of the loss itself: spread over perturbations at the last bit of H
    vals = []
    for _ in range(5):
        P = torch.as_tensor(rng.standard_normal((n, n)), device="cuda")
        vals.append(loss(Hd + 1e-15 * (0.5 * (P + P.T))[None], Sd))
    # no smaller than the rounding of the loss value itself: with |L| ~ 1e4 perturbations at
    # the last bit of H can leave every sample on the same float, so std() reads 0
    sigma = max(float(np.std(vals)), 2.0 ** -52 * abs(vals[0]))
    worst = 0.0
    for which, grad in (("H", Hb), ("S", Sb)):
        gnorm = float(torch.linalg.norm(grad).item())
        for _ in range(ndir):
            G = torch.as_tensor(rng.standard_normal((n, n)), device="cuda")
            G = 0.5 * (G + G.T)
            G /= torch.linalg.norm(G)
            D = (Lc @ G @ Lc.T)[None]
            D = 0.5 * (D + D.transpose(-1, -2))
            if which == "H":
                f = lambda t: loss(Hd + t * D, Sd)
            else:
                f = lambda t: loss(Hd, Sd + t * D)
            fd = (8.0 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12.0 * h)
            ad = float((grad * D).sum().item())
            # what a difference quotient can resolve: 1e-6 relative plus its own noise
            # (fourth-order weights: 18/12 of the loss noise over h)
            allow = gate * max(abs(fd), abs(ad)) + 20.0 * sigma / h
            worst = max(worst, abs(fd - ad) / allow)
    assert worst <= 1.0, (worst, sigma)


def test_adjoint_finite_differences(ctx):
    """64 + 64 directions at n = 400, h = 2e-4."""
    _fd_check(ctx, 400, 64, 2e-4, 1e-6, 400)


def test_adjoint_finite_differences_at_config_size(ctx):
    """n = 2808, the 216-atom size, 16 + 16 directions, h = 1e-3."""
    _fd_check(ctx, 2808, 16, 1e-3, 1e-6, 2808)


def test_autograd_function(ctx):
    from paper_2606_09058_gb300.gks import GKSSolve
    H, S = I.random_pencil(60, 4, True, 10.0)
    Ht = _cuda(H[None]).requires_grad_(True)
    St = _cuda(S[None]).requires_grad_(True)
    eps, rho, e_band, mu = GKSSolve.apply(Ht, St, 0.1, 40.0)
    L = e_band.sum() + (rho.abs() ** 2).sum() + eps.sum()
    L.backward()
    sol = ctx.solve(_cuda(H[None]), _cuda(S[None]), 0.1, 40.0)
    Hb, Sb = ctx.adjoint(sol, _cuda(S[None]), 0.1, rho_bar=2.0 * sol.rho,
                         eps_bar=torch.ones_like(sol.eps), e_band_bar=1.0)
    assert torch.allclose(Ht.grad, Hb, rtol=1e-9, atol=1e-9 * Hb.abs().max().item())
    assert torch.allclose(St.grad, Sb, rtol=1e-9, atol=1e-9 * Sb.abs().max().item())


def test_autograd_recompute_matches_saved(ctx):
    """recompute=True (no eigenvectors kept; backward solves again) gives the same gradients
    bit for bit: the solve is deterministic."""
    from paper_2606_09058_gb300.gks import GKSSolve
    H, S = I.random_pencil(70, 5, True, 10.0)
    grads = []
    for rec in (False, True):
        Ht = _cuda(H[None]).requires_grad_(True)
        St = _cuda(S[None]).requires_grad_(True)
        eps, rho, e_band, mu = GKSSolve.apply(Ht, St, 0.1, 40.0, "collinear", None, rec)
        (e_band.sum() + (rho.abs() ** 2).sum() + eps.sum()).backward()
        grads.append((Ht.grad.clone(), St.grad.clone()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])
