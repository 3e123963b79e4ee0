"""Mixed precision (GKS_MIXED_SPLITBF16): single-precision tridiagonalization, 5-digit
back-transform products, Ogita-Aishima refinement with FP64-accurate products.  The refined
eigenpairs must pass the same oracle gates as the FP64 path, and the sweeps must take the
orthonormality defect from the single-precision start down to the FP64 floor."""
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


def _scaled(H, S, eps, C):
    nh, ns = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    cn = np.linalg.norm(C, axis=0)
    G = C.conj().T @ S @ C - np.eye(C.shape[1])
    orth = np.abs(G / np.outer(cn, cn) / ns).max()
    R = H @ C - (S @ C) * eps
    bwd = (np.linalg.norm(R, axis=0) / ((nh + np.abs(eps) * ns) * cn)).max()
    return orth, bwd


def _check(sol, p, spin="collinear"):
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, spin, p.kweights)
    eps, C, rho = sol.eps.cpu().numpy(), sol.C.cpu().numpy(), sol.rho.cpu().numpy()
    nk, M = eps.shape
    for k in range(nk):
        Sk = O.spinor_overlap(p.S[k].numpy()) if spin == "noncollinear" else p.S[k].numpy()
        Hk = p.H[k].numpy()
        beta = O.eig_condition(Hk, Sk, ref.eps[k], ref.C[k])
        assert np.all(np.diff(eps[k]) >= 0)
        assert np.all(np.abs(eps[k] - ref.eps[k]) <= np.maximum(1e-10, 8 * beta)), np.abs(eps[k] - ref.eps[k]).max()
        orth, bwd = _scaled(Hk, Sk, eps[k], C[k])
        assert orth <= 1e-12 * math.sqrt(M) and bwd <= 1e-12 * math.sqrt(M), (orth, bwd)
        d = np.abs(Sk @ (rho[k] - ref.rho[k]) @ Sk).max()
        assert d <= 1e-9 * max(1.0, beta.max() / 1e-10), d
    assert abs(sol.mu.item() - ref.mu) <= 1e-3 * p.kT
    return ref


def test_mixed_si_cluster_real(gks):
    p = I.collinear_gamma((2, 1, 1), 0, 0.01)
    ctx = gks.Context(0, precision="mixed")
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec)
    _check(sol, p)
    st = ctx.refine_stats()[:, 0]
    assert st.shape == (6,)
    # the orthonormality defect at the start of each sweep: from the single-precision start
    # it falls to the FP64 floor (row-sum bound, about M u) and stays there
    assert 1e-12 < st[0] < 1e-2, st
    assert st[-1] <= 1e-12 * p.n, st
    assert st[-1] < st[0]


def test_mixed_kbatch_complex(gks):
    p = I.periodic((1, 1, 1), 1, 0.01)
    ctx = gks.Context(0, precision="mixed")
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, kweights=torch.as_tensor(p.kweights).cuda())
    _check(sol, p)
    st = ctx.refine_stats().reshape(6, p.nk, 2)
    assert np.all(st[-1, :, 0] <= 1e-12 * p.n), st[:, :, 0]


def test_mixed_noncollinear(gks):
    p = I.noncollinear((1, 1, 1), 2, 0.01)
    ctx = gks.Context(0, precision="mixed")
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec, "noncollinear")
    _check(sol, p, "noncollinear")


def test_mixed_sweep_count(gks):
    """The sweep count is the option's; more sweeps keep the eigenpairs at the FP64 floor."""
    p = I.collinear_gamma((1, 1, 1), 0, 0.01)
    ctx = gks.Context(0, precision="mixed", refine_sweeps=8)
    sol = ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec)
    _check(sol, p)
    st = ctx.refine_stats()
    assert st.shape == (8, 2) and st[-1, 0] <= 1e-12 * p.n


def test_mixed_rejects_partial_spectrum(gks):
    ctx = gks.Context(0, precision="mixed", n_ev=10)
    p = I.collinear_gamma((1, 1, 1), 0, 0.01)
    with pytest.raises(gks.GKSError) as ei:
        ctx.solve(p.H.cuda(), p.S.cuda(), p.kT, p.n_elec)
    assert ei.value.code == gks.GKS_EINVAL
