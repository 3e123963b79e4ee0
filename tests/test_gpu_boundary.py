"""The C-ABI options and entry points beyond the plain solve, through the binding:
reuse of the S factor, eigenpairs kept for the adjoint, eigen-only solves with gks_occupy
(shared mu across separately solved k-points, density and energy-density matrices),
partial spectrum (n_ev), spin-polarized runs, bounded waits that expire, the autotune
cache file and the precision options."""
import math
import os

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


def _scaled(H, S, eps, C):
    nh, ns = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    cn = np.linalg.norm(C, axis=0)
    G = C.conj().T @ S @ C - np.eye(C.shape[1])
    orth = np.abs(G / np.outer(cn, cn) / ns).max()
    R = H @ C - (S @ C) * eps
    bwd = (np.linalg.norm(R, axis=0) / ((nh + np.abs(eps) * ns) * cn)).max()
    return orth, bwd


def test_reuse_s_factor_bit_equal_and_skips_cholesky(gks):
    p = I.periodic((1, 1, 1), 1, 0.01)
    H1, S = p.H.cuda(), p.S.cuda()
    H2 = (p.H + 1e-3 * p.S).cuda()  # a new H with the same S (an SCF step)
    kw = torch.as_tensor(p.kweights).cuda()
    ctx = gks.Context(0, profile=True)
    ctx.solve(H1, S, p.kT, p.n_elec, kweights=kw)
    ctx.profile()
    reused = ctx.solve(H2, S, p.kT, p.n_elec, kweights=kw, reuse_s=True)
    names = {e["name"] for e in ctx.profile()}
    assert "stage:potrf" not in names and "stage:hegst" in names
    fresh = gks.Context(0).solve(H2, S, p.kT, p.n_elec, kweights=kw)
    for a, b in ((reused.eps, fresh.eps), (reused.C, fresh.C), (reused.rho, fresh.rho), (reused.mu, fresh.mu)):
        assert torch.equal(a, b)
    # a different S array is factored again
    S2 = S.clone()
    ctx.solve(H2, S2, p.kT, p.n_elec, kweights=kw, reuse_s=True)
    assert "stage:potrf" in {e["name"] for e in ctx.profile()}


def test_saved_eigenpairs_feed_the_adjoint(gks):
    p = I.collinear_gamma((1, 1, 1), 0, 0.01)
    ctx = gks.Context(0)
    H, S = p.H.cuda(), p.S.cuda()
    sol = ctx.solve(H, S, p.kT, p.n_elec, save_for_backward=True)
    rb = torch.randn_like(sol.rho)
    rb = rb + rb.transpose(-1, -2)
    ref = ctx.adjoint(sol, S, p.kT, rho_bar=rb)
    sol.C.zero_()  # the caller may overwrite its outputs: the context holds copies
    sol.eps.zero_()
    got = ctx.adjoint(None, S, p.kT, rho_bar=rb, complex_=False)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_eigen_only_and_occupy_reproduce_the_solve(gks):
    """gks_occupy on the solve's own eigenvalues returns its mu and rho bit for bit; k-points
    solved in two separate eigen-only calls (as two processes would) give the same mu and
    rho within the parity gates."""
    p = I.periodic((1, 1, 1), 1, 0.01)
    H, S = p.H.cuda(), p.S.cuda()
    kw = torch.as_tensor(p.kweights).cuda()
    ctx = gks.Context(0)
    full = ctx.solve(H, S, p.kT, p.n_elec, kweights=kw)
    mu, rho, eb, edm = ctx.occupy(full.eps, full.C, p.kT, p.n_elec, kweights_all=kw, edm=True)
    assert torch.equal(mu, full.mu) and torch.equal(rho, full.rho) and torch.equal(eb, full.e_band)
    # two "ranks": k-points 0..3 and 4..7, eigen-only, then the shared mu from all eps
    half = p.nk // 2
    parts = [ctx.solve(H[a:b].contiguous(), S[a:b].contiguous(), p.kT, p.n_elec, eigen_only=True)
             for a, b in ((0, half), (half, p.nk))]
    eps_all = torch.cat([q.eps for q in parts]).contiguous()
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, kweights=p.kweights)
    for r, q, k0 in ((0, parts[0], 0), (1, parts[1], half)):
        mu_r, rho_r, eb_r, edm_r = ctx.occupy(eps_all, q.C, p.kT, p.n_elec, k0=k0, kweights_all=kw, edm=True)
        assert abs(mu_r.item() - ref.mu) <= 1e-3 * p.kT
        for j in range(q.C.shape[0]):
            k = k0 + j
            Sk = p.S[k].numpy()
            beta = O.eig_condition(p.H[k].numpy(), Sk, ref.eps[k], ref.C[k])
            gate = 1e-9 * max(1.0, beta.max() / 1e-10)
            assert np.abs(Sk @ (rho_r[j].cpu().numpy() - ref.rho[k]) @ Sk).max() <= gate
            E_ref = O.energy_density_matrix(ref.C[k], ref.occ[k], ref.eps[k], 2.0)
            scale = max(1.0, np.abs(ref.eps[k][ref.occ[k] >= 1e-16]).max())
            assert np.abs(Sk @ (edm_r[j].cpu().numpy() - E_ref) @ Sk).max() <= gate * scale
    # the energy-density matrix of the full solve: tr(E S) = sum g_s f eps per k
    for k in range(p.nk):
        Sk = p.S[k].numpy()
        tr = np.trace(edm[k].cpu().numpy() @ Sk).real
        f = O.fermi((full.eps[k].cpu().numpy() - mu.item()) / p.kT)
        assert abs(tr - 2.0 * np.sum(f * full.eps[k].cpu().numpy())) <= 1e-8 * max(1.0, abs(tr))


@pytest.mark.parametrize("cplx", [False, True])
def test_partial_spectrum(gks, cplx):
    """n_ev eigenvectors: C is (nk, M, n_ev); eps, mu and rho as with all of them."""
    p = I.collinear_gamma((2, 1, 1), 0, 0.01) if not cplx else I.periodic((1, 1, 1), 1, 0.01)
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, kweights=p.kweights)
    n_ev = int(ref.n_rho.max()) + 7
    ctx = gks.Context(0, n_ev=n_ev)
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, kweights=torch.as_tensor(p.kweights).cuda())
    assert tuple(sol.C.shape) == (p.nk, p.M, n_ev)
    for k in range(p.nk):
        Hk, Sk = p.H[k].numpy(), p.S[k].numpy()
        beta = O.eig_condition(Hk, Sk, ref.eps[k], ref.C[k])
        eps = sol.eps[k].cpu().numpy()
        assert np.all(np.abs(eps - ref.eps[k]) <= np.maximum(1e-10, 8 * beta))
        orth, bwd = _scaled(Hk, Sk, eps[:n_ev], sol.C[k].cpu().numpy())
        assert orth <= 1e-12 * math.sqrt(p.M) and bwd <= 1e-12 * math.sqrt(p.M)
        assert np.abs(Sk @ (sol.rho[k].cpu().numpy() - ref.rho[k]) @ Sk).max() <= 1e-9 * max(1.0, beta.max() / 1e-10)
    # fewer eigenvectors than occupied states: a device-side GKS_EINVAL, context usable
    small = gks.Context(0, n_ev=int(ref.n_rho.min()) - 5)
    with pytest.raises(gks.GKSError) as ei:
        small.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, kweights=torch.as_tensor(p.kweights).cuda())
    assert ei.value.code == gks.GKS_EINVAL and "n_ev" in str(ei.value)


def test_spin_polarized_matches_oracle(gks):
    p = I.spin_polarized((2, 1, 1), 7, 0.01)
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, spin="spin_polarized")
    ctx = gks.Context(0)
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, spin="spin_polarized")
    assert tuple(sol.eps.shape) == (1, 2, p.n) and tuple(sol.rho.shape) == (1, 2, p.n, p.n)
    S = p.S[0].numpy()
    tr = 0.0
    for s_ in range(2):
        H = p.H[0, s_].numpy()
        beta = O.eig_condition(H, S, ref.eps[0, s_], ref.C[0, s_])
        assert np.all(np.abs(sol.eps[0, s_].cpu().numpy() - ref.eps[0, s_]) <= np.maximum(1e-10, 8 * beta))
        rho = sol.rho[0, s_].cpu().numpy()
        assert np.abs(S @ (rho - ref.rho[0, s_]) @ S).max() <= 1e-9 * max(1.0, beta.max() / 1e-10)
        tr += np.trace(rho @ S).real
    assert abs(tr - p.n_elec) <= 1e-9 * p.n_elec * 1e3
    assert abs(sol.mu.item() - ref.mu) <= 1e-3 * p.kT
    # the adjoint through a spin-polarized solve: the free-energy identity dF/dH = rho
    f = O.fermi((sol.eps.cpu().numpy() - sol.mu.item()) / p.kT)
    Hb, Sb = ctx.adjoint(sol, p.S.cuda(), p.kT, spin="spin_polarized",
                         eps_bar=torch.as_tensor(f).cuda().contiguous())
    for s_ in range(2):
        d = np.abs(S @ (Hb[0, s_].cpu().numpy() - sol.rho[0, s_].cpu().numpy()) @ S).max()
        assert d <= 1e-9 * np.abs(S @ sol.rho[0, s_].cpu().numpy() @ S).max()
    assert tuple(Sb.shape) == (1, p.n, p.n)


def test_bounded_wait_expires_and_the_context_recovers(gks):
    """A product whose operand copy never arrives: every CTA's bounded wait expires, the
    kernel frees its tensor memory and returns, gks_sync reports GKS_ETIMEOUT; the next
    solve on the same context passes parity."""
    ctx = gks.Context(0, debug=gks.GKS_DEBUG_SKIP_COPY, wait_limit=1 << 22)
    A = torch.randn(512, 512, dtype=torch.float64, device="cuda")
    C = torch.zeros(512, 512, dtype=torch.float64, device="cuda")
    with pytest.raises(gks.GKSError) as ei:
        ctx.gemm(A, A, C, mode="split")
    assert ei.value.code == gks.GKS_ETIMEOUT
    p = I.collinear_gamma((1, 1, 1), 0, 0.01)
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec)
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec)
    beta = O.eig_condition(p.H[0].numpy(), p.S[0].numpy(), ref.eps[0], ref.C[0])
    assert np.all(np.abs(sol.eps[0].cpu().numpy() - ref.eps[0]) <= np.maximum(1e-10, 8 * beta))
    # and a split product on the same context is whole again
    ctx.gemm(A, A, C, mode="split")
    assert torch.allclose(C, A @ A, rtol=0, atol=1e-10 * float((A.abs() @ A.abs()).max()))


def test_autotune_cache_file_round_trip(gks, tmp_path):
    path = str(tmp_path / "widths.txt")
    c1 = gks.Context(0, autotune_cache=path)
    c1.tune_set(700, True, "collinear", 192)
    c1.tune_set(3000, False, "noncollinear", 384)
    assert os.path.exists(path)
    c2 = gks.Context(0, autotune_cache=path)
    assert c2.tune_get(700, True, "collinear") == 192
    assert c2.tune_get(3000, False, "noncollinear") == 384


def test_precision_options(gks):
    with pytest.raises(gks.GKSError) as ei:
        gks.Context(0, precision="mixed_tf32")
    assert ei.value.code == gks.GKS_ENOTIMPL


def test_unknown_flags_rejected(gks):
    p = I.chain(20, 0.0, -1.0)
    H, S = (torch.as_tensor(x)[None].cuda() for x in p)
    ctx = gks.Context(0)
    eps = torch.empty(1, 20, dtype=torch.float64, device="cuda")
    C = torch.empty(1, 20, 20, dtype=torch.float64, device="cuda")
    rc = ctx._lib.gks_solve(ctx._h, gks._ptr(H), gks._ptr(S), 20, 1, 0, 0, 0.1, 10.0, None, 64, gks._ptr(eps),
                            gks._ptr(C), gks._ptr(torch.empty(1, dtype=torch.float64, device="cuda")),
                            gks._ptr(torch.empty_like(C)), None)
    assert rc == gks.GKS_EINVAL
