"""Parity at the workloads' own sizes, in the launch configuration the benchmark times.

* 512-atom k-batch (N = 6656, 8 k-points, complex128, shared mu): every column of every
  k-point checked for S-orthonormality and backward error (scaled gates), the density
  matrix checked against C diag(g_s f) C^H and Tr(rho S), time-reversal pairs
  eps(k) = eps(-k), every k-point's eigenvalues against the oracle's within
  max(1e-10, 8 beta_i); k-point 0 solved as a pencil of its own and compared with the
  oracle (eps, S rho S on sampled entries within the S-covariant gate, mu, E_band).
* 384-atom noncollinear cluster (2N = 9984): the same property checks, and eps, S rho S
  on sampled entries and mu against the oracle.
* The 48 uneven systems, solved in one batched launch sequence as the benchmark does:
  each compared with the oracle (eps and S rho S).
* The 216-atom cluster (N = 2808): the adjoint against central finite differences on 64 H
  and 64 S directions D = L G L^T, h = 1e-6.

Oracle results: the 512- and 384-atom ones are stored (tests/golden/make_fullsize.py, hours
of oracle time on the host cores; the pencils there are built on the CPU and agree with
the GPU-built ones here to a few rounding units, first-order inside the beta_i gates); the
48 systems' come from a background process started when the session collected these tests
(fullsize_support).  The property checks use FP64 products in torch."""
import math
import os

import numpy as np
import pytest
import torch

import fullsize_support as FS
from oracle import oracle as O
from paper_2606_09058_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def gks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_09058_gb300 import gks as g
    if not FS.started():
        FS.start()
    return g


def _norm2(A, iters=200):
    """||A||_2 of a Hermitian device matrix by power iteration (a lower bound: tighter gates)."""
    g = torch.Generator(device=A.device).manual_seed(1)
    v = torch.randn(A.shape[0], dtype=torch.float64, device=A.device, generator=g).to(A.dtype)
    v /= torch.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = A @ v
        lam = float(torch.linalg.norm(w))
        v = w / lam
    return lam


def _properties(H, S, eps, C, rho, gs, mu, kT):
    """Scaled orthonormality and backward error of every column (gates 1e-12 sqrt(M)), rho
    against C diag(g_s f) C^H (S-covariant: max |S (rho - ref) S|), tr(rho S).
    Returns (orth, bwd, drho, trace, beta) with beta the condition numbers from C."""
    M = H.shape[0]
    nh, ns = _norm2(H), _norm2(S)
    cn = torch.linalg.norm(C, dim=0)
    SC = S @ C
    G = C.conj().T @ SC
    G.diagonal().sub_(1.0)
    orth = float((G.abs() / torch.outer(cn, cn)).max()) / ns
    del G
    R = H @ C - SC * eps[None, :]
    bwd = float((torch.linalg.norm(R, dim=0) / ((nh + eps.abs() * ns) * cn)).max())
    del R, SC
    f = torch.as_tensor(O.fermi((eps.cpu().numpy() - mu) / kT), device=C.device)
    keep = f >= 1e-16
    Ck = C[:, keep]
    ref = (Ck * (gs * f[keep]).to(C.dtype)[None, :]) @ Ck.conj().T
    drho = float((S @ (rho - ref) @ S).abs().max())
    trace = float(torch.einsum("ij,ji->", rho, S).real)
    beta = (2.0 ** -53) * (nh + eps.abs() * ns) * cn ** 2
    return orth, bwd, drho, trace, beta.cpu().numpy()


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}_oracle.npz")
    if not os.path.exists(path):
        pytest.fail(f"{path} missing: written by tests/golden/make_fullsize.py")
    return np.load(path)


def _sampled_srs(S, rho, i, j):
    """(S rho S)[i, j] on the sampled pairs."""
    ii = torch.as_tensor(i.astype(np.int64), device=S.device)
    jj = torch.as_tensor(j.astype(np.int64), device=S.device)
    A = S[ii, :] @ rho
    return torch.einsum("pk,kp->p", A, S[:, jj]).cpu().numpy()


def test_kbatch512_full_size(gks):
    kb = I.workload("kbatch512", device="cuda")
    M, nk = kb.M, kb.nk
    kw = torch.as_tensor(np.asarray(kb.kweights, float)).cuda()
    ctx = gks.Context(0)
    sol = ctx.solve(kb.H, kb.S, kb.kT, kb.n_elec, kweights=kw)
    mu = float(sol.mu.item())
    tr = 0.0
    betas = []
    for k in range(nk):
        orth, bwd, drho, trace, beta = _properties(kb.H[k], kb.S[k], sol.eps[k], sol.C[k], sol.rho[k], 2.0, mu,
                                                   kb.kT)
        assert orth <= 1e-12 * math.sqrt(M), (k, orth)
        assert bwd <= 1e-12 * math.sqrt(M), (k, bwd)
        assert drho <= 1e-9 * max(1.0, beta.max() / 1e-10), (k, drho)
        assert torch.equal(sol.rho[k], sol.rho[k].conj().T)
        tr += kb.kweights[k] * trace
        betas.append(beta)
    bmax = max(b.max() for b in betas)
    assert abs(tr - kb.n_elec) <= 1e-9 * kb.n_elec * max(1.0, bmax / 1e-10)
    # time reversal: H(-k) = conj H(k), so the 8 Monkhorst-Pack points form 4 pairs
    kf = kb.meta["kpoints"]
    eps = sol.eps.cpu().numpy()
    for a in range(nk):
        b = int(np.argmin(np.abs(kf + kf[a]).sum(1)))
        assert b == nk - 1 - a
        assert np.all(np.abs(eps[a] - eps[b]) <= np.maximum(1e-10, 16 * np.maximum(betas[a], betas[b])))
    # every k-point's eigenvalues against the oracle's (k-points 0..3 stored; -k shares k's)
    g = _golden("kbatch512")
    for a in range(nk):
        r = a if a < 4 else nk - 1 - a
        tol = np.maximum(1e-10, 8 * g[f"beta{r}"])
        assert np.all(np.abs(eps[a] - g[f"eps{r}"]) <= tol), (a, np.abs(eps[a] - g[f"eps{r}"]).max())
    del sol
    # k-point 0 as a pencil of its own (its own mu), element by element against the oracle
    one = ctx.solve(kb.H[:1], kb.S[:1], kb.kT, kb.n_elec)
    e1 = one.eps[0].cpu().numpy()
    assert np.all(np.abs(e1 - g["eps0"]) <= np.maximum(1e-10, 8 * g["beta0"]))
    srs = _sampled_srs(kb.S[0], one.rho[0], g["k0_i"], g["k0_j"])
    gate = 1e-9 * max(1.0, g["beta0"].max() / 1e-10)
    assert np.abs(srs - g["k0_srs"]).max() <= gate, (np.abs(srs - g["k0_srs"]).max(), gate)
    assert abs(one.mu.item() - float(g["k0_mu"])) <= 1e-3 * kb.kT
    assert abs(one.e_band.item() - float(g["k0_eb"])) <= 1e-9 * abs(float(g["k0_eb"])) * max(1.0, g["beta0"].max() / 1e-10)


def test_nc384_full_size(gks):
    p = I.workload("nc384", device="cuda")
    ctx = gks.Context(0)
    sol = ctx.solve(p.H, p.S, p.kT, p.n_elec, spin="noncollinear")
    n = p.n
    S_nc = torch.zeros(2 * n, 2 * n, dtype=torch.complex128, device="cuda")
    S_nc[:n, :n] = p.S[0]
    S_nc[n:, n:] = p.S[0]
    orth, bwd, drho, trace, beta = _properties(p.H[0], S_nc, sol.eps[0], sol.C[0], sol.rho[0], 1.0,
                                               float(sol.mu.item()), p.kT)
    M = 2 * n
    assert orth <= 1e-12 * math.sqrt(M), orth
    assert bwd <= 1e-12 * math.sqrt(M), bwd
    assert drho <= 1e-9 * max(1.0, beta.max() / 1e-10), drho
    assert abs(trace - p.n_elec) <= 1e-9 * p.n_elec * max(1.0, beta.max() / 1e-10)
    g = _golden("nc384")
    e = sol.eps[0].cpu().numpy()
    assert np.all(np.abs(e - g["eps"]) <= np.maximum(1e-10, 8 * g["beta"])), np.abs(e - g["eps"]).max()
    srs = _sampled_srs(S_nc, sol.rho[0], g["i"], g["j"])
    gate = 1e-9 * max(1.0, g["beta"].max() / 1e-10)
    assert np.abs(srs - g["srs"]).max() <= gate, (np.abs(srs - g["srs"]).max(), gate)
    assert abs(sol.mu.item() - float(g["mu"])) <= 1e-3 * p.kT


def test_uneven48_all_systems_against_oracle(gks):
    probs = FS.inputs("uneven48")
    stream = torch.cuda.Stream()
    ctx = gks.Context(0, stream)
    items = [dict(H=p.H.contiguous(), S=p.S.contiguous(), kT=p.kT, n_elec=p.n_elec, spin=p.spin) for p in probs]
    with torch.cuda.stream(stream):
        sols = ctx.solve_batched(items, nstreams=8)
    torch.cuda.synchronize()
    ref = FS.oracle_result("u")
    for b, (p, s) in enumerate(zip(probs, sols)):
        eps = s.eps[0].cpu().numpy()
        beta = ref[f"beta{b}"]
        assert np.all(np.abs(eps - ref[f"eps{b}"]) <= np.maximum(1e-10, 8 * beta)), (b, np.abs(eps - ref[f"eps{b}"]).max())
        S = p.S[0]
        if p.spin == "noncollinear":
            n = p.n
            Sn = torch.zeros(2 * n, 2 * n, dtype=torch.complex128, device="cuda")
            Sn[:n, :n] = S
            Sn[n:, n:] = S
            S = Sn
        srs = (S @ s.rho[0] @ S).cpu().numpy()
        gate = 1e-9 * max(1.0, beta.max() / 1e-10)
        assert np.abs(srs - ref[f"srs{b}"]).max() <= gate, (b, np.abs(srs - ref[f"srs{b}"]).max(), gate)
        assert abs(s.mu.item() - float(ref[f"mu{b}"])) <= 1e-3 * p.kT, b


def test_adjoint216_finite_differences(gks):
    """The 216-atom cluster (N = 2808, kT 0.02, n_elec 864): loss E_band + ||rho - rho_t||^2
    with rho_t the density matrix of H + 1e-3 S U2 S.  Central differences (h = 1e-6) along
    64 H and 64 S directions D = L G L^T against the adjoint: relative agreement 1e-6 plus
    the quotient's own rounding noise (20 sigma / h, sigma the measured noise of the loss)."""
    p = I.workload("adjoint216", device="cuda")
    H, S = p.H, p.S
    n = p.n
    rng = np.random.default_rng(9058004)
    U2 = rng.uniform(-1.0, 1.0, (n, n))
    U2 = torch.as_tensor(0.5 * (U2 + U2.T), device="cuda")
    ctx = gks.Context(0)
    rho_t = ctx.solve((H[0] + 1e-3 * S[0] @ U2 @ S[0])[None].contiguous(), S, p.kT, p.n_elec).rho.clone()
    base = ctx.solve(H, S, p.kT, p.n_elec)

    def loss(Hx, Sx):
        s = ctx.solve(Hx, Sx, p.kT, p.n_elec)
        return float(s.e_band.item() + ((s.rho - rho_t) ** 2).sum().item())

    Hb, Sb = ctx.adjoint(base, S, p.kT, rho_bar=2.0 * (base.rho - rho_t), e_band_bar=1.0)
    Lc = torch.linalg.cholesky(S[0])
    vals = []
    for _ in range(5):
        P = torch.as_tensor(rng.standard_normal((n, n)), device="cuda")
        vals.append(loss(H + 1e-15 * (0.5 * (P + P.T))[None], S))
    sigma = max(float(np.std(vals)), 2.0 ** -52 * abs(vals[0]))
    h = 1e-6
    worst = 0.0
    for which, grad in (("H", Hb), ("S", Sb)):
        for _ in range(64):
            G = torch.as_tensor(rng.standard_normal((n, n)), device="cuda")
            G = 0.5 * (G + G.T)
            G /= torch.linalg.norm(G)
            D = (Lc @ G @ Lc.T)[None]
            D = 0.5 * (D + D.transpose(-1, -2))
            if which == "H":
                fd = (loss(H + h * D, S) - loss(H - h * D, S)) / (2.0 * h)
            else:
                fd = (loss(H, S + h * D) - loss(H, S - h * D)) / (2.0 * h)
            ad = float((grad * D).sum().item())
            allow = 1e-6 * max(abs(fd), abs(ad)) + 20.0 * sigma / h
            worst = max(worst, abs(fd - ad) / allow)
    assert worst <= 1.0, (worst, sigma)
