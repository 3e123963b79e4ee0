"""The Loewdin reduction (paper Sec. 3.1 Parts 2-1 .. 2-5: eig S, V = U s^-1/2,
H' = V^H H V, C = V C') through the C ABI, against the oracle: raw gates on well-conditioned
pencils (where both reductions are accurate), and on the Si cluster against the oracle's
own Loewdin route with the condition-scaled gates; the kept factor V is reused."""
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
    return gks.Context(0, reduction="lowdin")


def _scaled(H, S, eps, C):
    nh, ns = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    cn = np.linalg.norm(C, axis=0)
    G = C.conj().T @ S @ C - np.eye(C.shape[1])
    orth = np.abs(G / np.outer(cn, cn) / ns).max()
    R = H @ C - (S @ C) * eps
    bwd = (np.linalg.norm(R, axis=0) / ((nh + np.abs(eps) * ns) * cn)).max()
    return orth, bwd


@pytest.mark.parametrize("cplx,m", [(False, 150), (True, 130), (False, 389), (True, 300)])
def test_lowdin_random_pencil_raw_gates(ctx, cplx, m):
    H, S = I.random_pencil(m, 800 + m, cplx, cond=1e2)
    sol = ctx.solve(torch.as_tensor(H)[None].cuda(), torch.as_tensor(S)[None].cuda(), 0.1, 0.6 * m)
    ref = O.solve(H[None], S[None], 0.1, 0.6 * m)
    eps, C, rho = sol.eps[0].cpu().numpy(), sol.C[0].cpu().numpy(), sol.rho[0].cpu().numpy()
    assert np.abs(eps - ref.eps[0]).max() <= 1e-10 * max(1.0, np.abs(ref.eps[0]).max())
    orth, bwd = _scaled(H, S, eps, C)
    assert orth <= 1e-12 * math.sqrt(m) and bwd <= 1e-12 * math.sqrt(m), (orth, bwd)
    assert np.abs(S @ (rho - ref.rho[0]) @ S).max() <= 1e-9
    # mu inside a wide gap is ill-determined (its bracket is flat): check the electron count
    # it gives on the oracle's eigenvalues instead
    count = 2.0 * O.fermi((ref.eps[0] - sol.mu.item()) / 0.1).sum()
    assert abs(count - 0.6 * m) <= 1e-9 * m


@pytest.mark.parametrize("tiling", [(1, 1, 1), (2, 1, 1)])
def test_lowdin_si_cluster_against_oracle_lowdin(ctx, tiling):
    p = I.collinear_gamma(tiling, 0, 0.01)
    H, S = p.H.numpy(), p.S.numpy()
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec)
    ref = O.solve(H, S, p.kT, p.n_elec, reduction="lowdin")
    beta = O.eig_condition(H[0], S[0], ref.eps[0], ref.C[0])
    eps = sol.eps[0].cpu().numpy()
    assert np.all(np.abs(eps - ref.eps[0]) <= np.maximum(1e-10, 8 * beta)), np.abs(eps - ref.eps[0]).max()
    d = np.abs(S[0] @ (sol.rho[0].cpu().numpy() - ref.rho[0]) @ S[0]).max()
    assert d <= 1e-9 * max(1.0, beta.max() / 1e-10), d


def test_lowdin_reuses_its_factor(ctx):
    from paper_2606_09058_gb300 import gks
    p = I.periodic((1, 1, 1), 1, 0.01)
    H2 = (p.H + 1e-3 * p.S).cuda()
    S = p.S.cuda()
    c = gks.Context(0, reduction="lowdin", profile=True)
    c.solve(p.H.cuda(), S, p.kT, p.n_elec)
    c.profile()
    again = c.solve(H2, S, p.kT, p.n_elec, reuse_s=True)
    assert "stage:potrf" not in {e["name"] for e in c.profile()}
    fresh = gks.Context(0, reduction="lowdin").solve(H2, S, p.kT, p.n_elec)
    assert torch.equal(again.eps, fresh.eps) and torch.equal(again.rho, fresh.rho)


def test_lowdin_noncollinear_not_implemented(ctx):
    from paper_2606_09058_gb300 import gks
    p = I.noncollinear((1, 1, 1), 2, 0.01)
    with pytest.raises(gks.GKSError) as ei:
        ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, "noncollinear")
    assert ei.value.code == gks.GKS_ENOTIMPL
