"""Control flow of the GKSSolve autograd Function on the CPU, with a stand-in context in
place of the CUDA library: with recompute=True the eigenvectors are not saved and backward
solves the same inputs again before the adjoint; both modes return the adjoint's arrays."""
import torch

from paper_2606_09058_gb300 import gks


class _FakeContext:
    def __init__(self):
        self.solves = []
        self.adjoints = []
        self.width = 256

    def tune_get(self, n, complex_=False, spin="collinear"):
        return self.width

    def solve(self, H, S, kT, n_elec, spin="collinear", kweights=None):
        self.solves.append((H.data_ptr(), S.data_ptr(), kT, n_elec, spin, kweights))
        nk, M = H.shape[0], H.shape[1]
        eps = torch.arange(M, dtype=torch.float64).repeat(nk, 1)
        C = torch.eye(M, dtype=H.dtype).repeat(nk, 1, 1) * 2.0
        return gks.Solution(eps, C, torch.zeros(1, dtype=torch.float64), C.clone(), torch.ones(1, dtype=torch.float64))

    def adjoint(self, sol, S, kT, spin, kweights, rho_bar=None, eps_bar=None, e_band_bar=0.0):
        self.adjoints.append((sol.C.clone(), sol.eps.clone(), e_band_bar))
        nk, M = sol.C.shape[0], sol.C.shape[1]
        return torch.full((nk, M, M), 3.0, dtype=sol.C.dtype), torch.full(S.shape, 5.0, dtype=sol.C.dtype)


def _run(monkeypatch, recompute):
    fake = _FakeContext()
    monkeypatch.setattr(gks, "context", lambda device=None: fake)
    H = torch.randn(1, 4, 4, dtype=torch.float64, requires_grad=True)
    S = torch.randn(1, 4, 4, dtype=torch.float64, requires_grad=True)
    eps, rho, e_band, mu = gks.GKSSolve.apply(H, S, 0.1, 2.0, "collinear", None, recompute)
    (rho.sum() + e_band.sum() + eps.sum()).backward()
    return fake, H.grad, S.grad


def test_saved_eigenvectors(monkeypatch):
    fake, gH, gS = _run(monkeypatch, False)
    assert len(fake.solves) == 1 and len(fake.adjoints) == 1
    assert torch.equal(gH, torch.full((1, 4, 4), 3.0, dtype=torch.float64))
    assert torch.equal(gS, torch.full((1, 4, 4), 5.0, dtype=torch.float64))


def test_recompute_solves_again_with_the_same_inputs(monkeypatch):
    fake, gH, gS = _run(monkeypatch, True)
    assert len(fake.solves) == 2 and fake.solves[0] == fake.solves[1]
    assert len(fake.adjoints) == 1 and fake.adjoints[0][2] == 1.0
    assert torch.equal(fake.adjoints[0][0], torch.eye(4, dtype=torch.float64)[None] * 2.0)
    assert torch.equal(gH, torch.full((1, 4, 4), 3.0, dtype=torch.float64))
    assert torch.equal(gS, torch.full((1, 4, 4), 5.0, dtype=torch.float64))


def test_recompute_refuses_a_changed_width(monkeypatch):
    """A tuned width set between forward and backward would change the recomputed C."""
    import pytest
    fake = _FakeContext()
    monkeypatch.setattr(gks, "context", lambda device=None: fake)
    H = torch.randn(1, 4, 4, dtype=torch.float64, requires_grad=True)
    S = torch.randn(1, 4, 4, dtype=torch.float64, requires_grad=True)
    eps, rho, e_band, mu = gks.GKSSolve.apply(H, S, 0.1, 2.0, "collinear", None, True)
    fake.width = 512
    with pytest.raises(RuntimeError, match="width"):
        rho.sum().backward()
