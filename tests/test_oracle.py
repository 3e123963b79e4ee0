"""Pins for the CPU oracle: closed forms, exact brute force, invariants and an
independent LAPACK cross-check.  Each test fixes something the oracle cannot know from
itself, chosen so that a dropped term, a wrong sign or index, or a transposed operand in
any stage fails at least one of them."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import oracle as O
from paper_2606_09058_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _match_columns(A, B):
    """max over columns of min(|a - b|, |a + b|) after unit-modulus phase alignment."""
    err = 0.0
    for j in range(A.shape[1]):
        a, b = A[:, j], B[:, j]
        ph = np.vdot(b, a)
        ph = ph / abs(ph) if abs(ph) > 0 else 1.0
        err = max(err, np.abs(a - ph * b).max())
    return err


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 7, 50, 161])
def test_chain_closed_form(n):
    """S = I chain: eps_j = e0 + 2t cos(j pi/(n+1)), c_ij = sqrt(2/(n+1)) sin(i j pi/(n+1))."""
    e0, t = 0.3, -1.0
    H, S = I.chain(n, e0, t)
    eps, C = O.eigh_generalized(H, S)
    j = np.arange(1, n + 1)
    ref = e0 + 2 * t * np.cos(j * np.pi / (n + 1))          # ascending for t < 0
    assert np.abs(eps - ref).max() <= 1e-13 * max(1, n)
    i = np.arange(1, n + 1)
    V = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, j) * np.pi / (n + 1))
    assert _match_columns(C, V) <= 1e-12 * max(1, n)


@pytest.mark.parametrize("n,s", [(5, 0.2), (40, -0.3), (120, 0.45)])
def test_generalized_chain_closed_form(n, s):
    """S tridiagonal (1, s): eps_j = (e0 + 2t cos th_j)/(1 + 2s cos th_j), th_j = j pi/(n+1)."""
    e0, t = -0.5, 0.7
    H, S = I.chain(n, e0, t, s)
    eps, C = O.eigh_generalized(H, S)
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    ref = np.sort((e0 + 2 * t * np.cos(th)) / (1 + 2 * s * np.cos(th)))
    assert np.abs(eps - ref).max() <= 1e-12 * max(1, np.abs(ref).max())
    assert np.abs(C.T @ S @ C - np.eye(n)).max() <= 1e-12


@pytest.mark.parametrize("n,phi", [(6, 0.3), (31, 1.1), (64, 2.5)])
def test_twisted_ring_closed_form(n, phi):
    """Complex Hermitian ring with H_{j,j+1} = t e^{i phi/n}: eps_m = e0 + 2t cos((2 pi m + phi)/n)."""
    e0, t = 0.1, 0.8
    H, S = I.twisted_ring(n, e0, t, phi)
    eps, C = O.eigh_generalized(H, S)
    ref = np.sort(e0 + 2 * t * np.cos((2 * np.pi * np.arange(n) + phi) / n))
    assert np.abs(eps - ref).max() <= 1e-13 * n
    assert np.abs(H @ C - C * eps).max() <= 1e-12 * n


# ------------------------------------------------------------------ exact brute force

def _rational_pencil(n, seed, cplx):
    import sympy as sp
    rng = np.random.default_rng(seed)
    def rat(x):
        return sp.Rational(int(x), 8)
    Hre = rng.integers(-16, 17, size=(n, n))
    Him = rng.integers(-16, 17, size=(n, n)) if cplx else np.zeros((n, n), int)
    B = rng.integers(-8, 9, size=(n, n))
    H = sp.zeros(n, n)
    for i in range(n):
        for j in range(i + 1):
            if i == j:
                H[i, i] = rat(Hre[i, i])
            else:
                v = rat(Hre[i, j]) + (sp.I * rat(Him[i, j]) if cplx else 0)
                H[i, j] = v
                H[j, i] = sp.conjugate(v)
    Bm = sp.Matrix(n, n, lambda i, j: rat(B[i, j]) + (sp.I * rat(B[j, i]) if cplx else 0))
    S = Bm * Bm.H + sp.eye(n)
    return H, S


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("cplx", [False, True])
def test_bruteforce_characteristic_roots(n, cplx):
    """Roots of det(H - lam S) in exact rational arithmetic (real symmetric, or complex
    Hermitian with Gaussian-rational entries), isolated and evaluated to 30 digits."""
    sp = pytest.importorskip("sympy")
    Hs, Ss = _rational_pencil(n, 1000 + n + (50 if cplx else 0), cplx)
    lam = sp.Symbol("lam")
    poly = sp.Poly(sp.expand((Hs - lam * Ss).det()), lam)
    coeffs = [sp.re(c) for c in poly.all_coeffs()]
    assert all(sp.im(c) == 0 for c in poly.all_coeffs())
    roots = sorted(float(r.evalf(30)) for r in sp.Poly(coeffs, lam).real_roots())
    assert len(roots) == n
    H = np.array(Hs.evalf(), dtype=complex if cplx else float)
    S = np.array(Ss.evalf(), dtype=complex if cplx else float)
    eps, C = O.eigh_generalized(H, S)
    scale = np.abs(np.array(roots)).max() + 1.0
    assert np.abs(eps - np.array(roots)).max() <= 1e-13 * scale
    assert np.abs(C.conj().T @ S @ C - np.eye(n)).max() <= 1e-13


# ------------------------------------------------------------------ each stage on its own

@pytest.mark.parametrize("cplx", [False, True])
def test_stage_cholesky(cplx):
    _, S = I.random_pencil(37, 5, cplx, cond=1e6)
    L = O.cholesky(S)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.all(np.real(np.diag(L)) > 0) and np.abs(np.imag(np.diag(L))).max() == 0
    assert np.abs(L @ L.conj().T - S).max() <= 1e-14 * np.abs(S).max() * 37
    # the Cholesky factor is unique: LAPACK's must agree
    assert np.abs(L - np.linalg.cholesky(S)).max() <= 1e-10


def test_stage_cholesky_reports_column():
    S = np.eye(6)
    S[3, 3] = -1.0
    with pytest.raises(O.OracleError, match="column 3"):
        O.cholesky(S)


@pytest.mark.parametrize("cplx", [False, True])
def test_stage_reduce(cplx):
    H, S = I.random_pencil(29, 7, cplx, cond=1e3)
    L = O.cholesky(S)
    Hp = O.reduce_standard(L, H)
    assert np.abs(Hp - Hp.conj().T).max() == 0
    assert np.abs(L @ Hp @ L.conj().T - H).max() <= 1e-12
    ref = sl.solve_triangular(L, sl.solve_triangular(L, H, lower=True).conj().T, lower=True)
    assert np.abs(Hp - ref).max() <= 1e-10


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 64])
def test_stage_tridiag_and_backtransform(cplx, n):
    H, _ = I.random_pencil(n, 11 + n, cplx)
    d, sub, U, beta = O.tridiagonalize(H)
    Q = np.eye(n, dtype=H.dtype)
    for k in range(n - 2):                       # Q = P_0 P_1 ... P_{n-3}
        u = U[k]
        Q = Q @ (np.eye(n) - beta[k] * np.outer(u, u.conj()))
    T = np.diag(d).astype(H.dtype)
    if n > 1:
        T += np.diag(sub, -1) + np.diag(sub.conj(), 1)
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 1e-13 * max(1, n)
    assert np.abs(Q @ T @ Q.conj().T - H).max() <= 1e-13 * max(1, n) * np.abs(H).max()
    lam, Z = O.tridiagonal_eig(d, np.abs(sub))
    X = O.back_transform(sub, U, beta, Z)
    assert np.abs(H @ X - X * lam).max() <= 1e-12 * max(1, n) * np.abs(H).max()
    assert np.abs(X.conj().T @ X - np.eye(n)).max() <= 1e-13 * max(1, n)


@pytest.mark.parametrize("kind", ["random", "wilkinson", "clustered", "split", "zero"])
def test_stage_tridiagonal_ql(kind):
    rng = np.random.default_rng(3)
    n = 60
    if kind == "random":
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
    elif kind == "wilkinson":                    # W+_n: pairs of eigenvalues agreeing to many digits
        n = 21
        d, e = np.abs(np.arange(n) - 10).astype(float), np.ones(n - 1)
    elif kind == "clustered":
        d, e = np.ones(n) + 1e-12 * rng.standard_normal(n), 1e-9 * rng.standard_normal(n - 1)
    elif kind == "split":
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
        e[[5, 20, 21, 40]] = 0.0
    else:
        d, e = np.zeros(n), np.zeros(n - 1)
    lam, Z = O.tridiagonal_eig(d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.all(np.diff(lam) >= 0)
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-13 * n
    assert np.abs(T @ Z - Z * lam).max() <= 1e-14 * n * max(1.0, np.abs(T).max())
    ref = sl.eigh_tridiagonal(d, e, eigvals_only=True)
    assert np.abs(lam - ref).max() <= 1e-13 * n * max(1.0, np.abs(T).max())


# ------------------------------------------------------------------ pencils and invariants

@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("cond", [1e1, 1e6, 1e10])
def test_lapack_cross_check(cplx, cond):
    """Independent LAPACK solve (Cholesky-based sygvd/hegvd).  A random H is not bounded
    relative to an ill-conditioned S, so ||H'|| = max|eps| >> ||H||/||S|| and both
    Cholesky-based solvers carry errors of order u ||S|| ||H'|| ||c_i||^2 (the two-sided
    reduction's backward error), which is the bound used here."""
    n = 48
    H, S = I.random_pencil(n, 21, cplx, cond)
    eps, C = O.eigh_generalized(H, S)
    ref = sl.eigh(H, S, eigvals_only=True)
    cn = np.sum(np.abs(C) ** 2, axis=0)
    bound = O.U_ROUND * (np.linalg.norm(H, 2) + np.abs(eps).max() * np.linalg.norm(S, 2)) * cn
    assert np.all(np.abs(eps - ref) <= np.maximum(1e-12, 8 * bound))


def _scaled_checks(H, S, eps, C):
    nh, ns = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    cn = np.linalg.norm(C, axis=0)
    G = C.conj().T @ S @ C - np.eye(C.shape[1])
    orth = np.abs(G / np.outer(cn, cn) / ns).max()
    R = H @ C - (S @ C) * eps
    bwd = (np.linalg.norm(R, axis=0) / ((nh + np.abs(eps) * ns) * cn)).max()
    return orth, bwd


@pytest.mark.parametrize("tiling", [(1, 1, 1), (2, 1, 1)])
def test_cluster_invariants(tiling):
    """Scaled S-orthonormality and backward error, and Tr(rho S) = n_elec, on the Si
    Gaussian basis (kappa(S) ~ 1e9 .. 1e10)."""
    p = I.collinear_gamma(tiling, 0, 0.01)
    H, S = p.H[0].numpy(), p.S[0].numpy()
    r = O.solve(H, S, p.kT, p.n_elec)
    orth, bwd = _scaled_checks(H, S, r.eps[0], r.C[0])
    M = H.shape[0]
    assert orth <= 1e-12 * math.sqrt(M)
    assert bwd <= 1e-12 * math.sqrt(M)
    tr = np.trace(r.rho[0] @ S).real
    beta = O.eig_condition(H, S, r.eps[0], r.C[0])
    assert abs(tr - p.n_elec) <= 1e-9 * p.n_elec * max(1.0, beta.max() / 1e-10)
    ref = sl.eigh(H, S, eigvals_only=True)
    assert np.all(np.abs(r.eps[0] - ref) <= np.maximum(1e-10, 8 * beta))
    # E_band = Tr(rho H) for a single k-point
    assert abs(r.e_band - np.trace(r.rho[0] @ H).real) <= 1e-9 * max(1.0, abs(r.e_band)) * max(1.0, beta.max() / 1e-10)


def test_kpoint_time_reversal_pairs():
    """H(-k) = conj H(k): the 8 Monkhorst-Pack points form 4 pairs with equal spectra."""
    p = I.periodic((1, 1, 1), 1, 0.01)
    kf = p.meta["kpoints"]
    r = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, kweights=p.kweights)
    for a in range(p.nk):
        b = int(np.argmin(np.abs(kf + kf[a]).sum(1)))
        assert np.allclose(kf[b], -kf[a])
        beta = O.eig_condition(p.H[a].numpy(), p.S[a].numpy(), r.eps[a], r.C[a])
        assert np.all(np.abs(r.eps[a] - r.eps[b]) <= np.maximum(1e-10, 16 * beta))
    tr = sum(p.kweights[k] * np.trace(r.rho[k] @ p.S[k].numpy()).real for k in range(p.nk))
    assert abs(tr - p.n_elec) <= 1e-6 * p.n_elec


def test_noncollinear_zero_mixing_doubles_collinear():
    """Delta = lambda = 0: every collinear eigenvalue appears exactly twice."""
    p = I.noncollinear((1, 1, 1), 2, 0.01, delta=0.0, lam=0.0)
    Hc, Sc = p.meta["H"].numpy(), p.meta["S"].numpy()
    ec, Cc = O.eigh_generalized(Hc, Sc)
    r = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, spin="noncollinear")
    beta = O.eig_condition(Hc, Sc, ec, Cc)
    assert np.all(np.abs(r.eps[0][0::2] - ec) <= np.maximum(1e-10, 16 * beta))
    assert np.all(np.abs(r.eps[0][1::2] - ec) <= np.maximum(1e-10, 16 * beta))


def test_noncollinear_collinear_moments_split():
    """All m parallel to z and lambda = 0: spec = spec(H + D Sz, S) U spec(H - D Sz, S)."""
    import torch
    p = I.noncollinear((1, 1, 1), 2, 0.01)
    H, S = p.meta["H"], p.meta["S"]
    natoms = p.meta["atoms"]
    m = np.zeros((natoms, 3))
    m[:, 2] = np.where(np.arange(natoms) % 3 == 0, -1.0, 1.0)
    HN = I.spinor_hamiltonian(H, S, m, p.meta["KA"], 0.05, 0.0).numpy()
    n = H.shape[0]
    r = O.solve(HN[None], S.numpy()[None].astype(complex), 0.01, 4.0 * natoms, spin="noncollinear")
    up = HN[:n, :n].real
    dn = HN[n:, n:].real
    assert np.abs(HN[:n, n:]).max() == 0
    eu, Cu = O.eigh_generalized(up, S.numpy())
    ed, Cd = O.eigh_generalized(dn, S.numpy())
    both = np.sort(np.concatenate([eu, ed]))
    beta = np.concatenate([O.eig_condition(up, S.numpy(), eu, Cu), O.eig_condition(dn, S.numpy(), ed, Cd)])
    assert np.all(np.abs(r.eps[0] - both) <= np.maximum(1e-10, 16 * beta.max()))


def test_noncollinear_uniform_chain_closed_form():
    """S = I chain with one uniform unit moment: eps = e0 + 2t cos th_j +- Delta."""
    n, e0, t, delta = 24, 0.2, -0.6, 0.05
    H, S = I.chain(n, e0, t)
    import torch
    m = np.array([[0.6, 0.0, 0.8]])
    HN = I.spinor_hamiltonian(torch.tensor(H), torch.tensor(S), m, np.zeros((1, n, n)), delta, 0.0,
                              block=n).numpy()
    r = O.solve(HN[None], S[None].astype(complex), 0.01, float(n), spin="noncollinear")
    base = e0 + 2 * t * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    ref = np.sort(np.concatenate([base + delta, base - delta]))
    assert np.abs(r.eps[0] - ref).max() <= 1e-13 * n


# ------------------------------------------------------------------ occupations and mu

def test_fermi_function():
    x = np.array([-800.0, -40.0, -1.0, 0.0, 1.0, 40.0, 800.0])
    f = O.fermi(x)
    assert f[3] == 0.5
    assert np.all(np.isfinite(f))
    assert np.abs(f + O.fermi(-x) - 1).max() <= 1e-16
    assert abs(f[4] - 1 / (1 + math.e)) <= 1e-16


def test_mu_particle_hole_symmetry():
    """Half-filled bipartite chain (e0 = 0): mu = 0 by particle-hole symmetry."""
    n = 40
    H, S = I.chain(n, 0.0, -1.0)
    r = O.solve(H, S, 0.05, float(n))
    assert abs(r.mu) <= 1e-12
    assert abs(np.trace(r.rho[0]).real - n) <= 1e-10


def test_mu_two_levels():
    """Two levels, one electron pair: f(e1 - mu) + f(e2 - mu) = 1 gives mu = (e1 + e2)/2."""
    H = np.diag([-0.3, 0.5])
    r = O.solve(H, np.eye(2), 0.07, 2.0)
    assert abs(r.mu - 0.1) <= 1e-14
    assert abs(r.occ[0].sum() - 1.0) <= 1e-14


def test_mu_rejects_bad_arguments():
    H = np.diag([-0.3, 0.5])
    with pytest.raises(O.OracleError):
        O.solve(H, np.eye(2), 0.0, 2.0)
    with pytest.raises(O.OracleError):
        O.solve(H, np.eye(2), 0.01, 4.0)


def test_density_matrix_convention_and_truncation():
    """rho = C diag(g_s f) C^H; the paper's n_lm = sum_i f_i c*_li c_mi equals conj(rho)/g_s."""
    H, S = I.random_pencil(12, 4, True, 10.0)
    r = O.solve(H, S, 0.5, 6.0)
    C, f = r.C[0], r.occ[0]
    n_paper = np.einsum("i,li,mi->lm", f, C.conj(), C)
    assert np.abs(n_paper - r.rho[0].conj() / 2.0).max() <= 1e-12
    assert np.abs(r.rho[0] - r.rho[0].conj().T).max() <= 1e-13


# ------------------------------------------------------------------ workload structure

def _golden():
    out = {}
    with open(os.path.join(GOLDEN, "paper_sizes.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def test_paper_workload_sizes():
    g = _golden()
    assert I.N_PER_ATOM == g["basis_per_atom"]
    assert abs(I.A_BOHR / 1.8897261 - g["lattice_angstrom"]) < 2e-3
    rng = np.random.default_rng(0)
    assert len(I.diamond_positions((5, 5, 6), rng)) == g["atoms_collinear_big"]
    assert g["atoms_collinear_big"] * I.N_PER_ATOM == g["basis_collinear_big"]
    assert len(I.diamond_positions((4, 4, 5), rng)) == g["atoms_nc_big"]
    assert g["atoms_nc_big"] * I.N_PER_ATOM == g["basis_nc_big"]
    n = 6656
    assert np.zeros((n, n), np.complex128).nbytes == g["bytes_per_complex_n2"] * n * n
    assert np.zeros((2 * n, 2 * n), np.complex128).nbytes == g["bytes_per_nc_n2"] * n * n
    assert len(I.mp_kpoints((2, 2, 2))) == g["kmesh"] ** 3


# ------------------------------------------------------------------ adjoint

def _loss_and_grads(H, S, kT, ne, spin, rt, a_eps):
    r = O.solve(H, S, kT, ne, spin)
    L = r.e_band + sum(np.sum(np.abs(r.rho[k] - rt[k]) ** 2) for k in range(r.rho.shape[0]))
    L += float(np.sum(a_eps * r.eps))
    return L, r


@pytest.mark.parametrize("case", ["real", "complex", "noncollinear"])
def test_adjoint_matches_finite_differences(case):
    """Central differences (h = 1e-5) along Hermitian directions D = L G L^H (G of unit
    Frobenius norm, L = chol S) agree with the hand adjoint to 1e-6 relative on
    well-conditioned pencils."""
    rng = np.random.default_rng(11)
    if case == "noncollinear":
        n = 10
        A = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
        H = (0.5 * (A + A.conj().T))[None]
        _, S = I.random_pencil(n, 12, True, 5.0)
        S = S[None]
        spin, kT, ne = "noncollinear", 0.3, 8.0
    else:
        H, S = I.random_pencil(18, 13, case == "complex", 10.0)
        H, S = H[None], S[None]
        spin, kT, ne = "collinear", 0.2, 14.0
    M = H.shape[1]
    rt = O.solve(H + 0.05 * np.eye(M)[None], S, kT, ne, spin).rho
    a_eps = rng.standard_normal((1, M)) * 0.1
    L0, r = _loss_and_grads(H, S, kT, ne, spin, rt, a_eps)
    Hb, Sb = O.adjoint(r, kT, spin, rho_bar=2 * (r.rho - rt), eps_bar=a_eps, e_band_bar=1.0)
    Lc = np.linalg.cholesky(S[0])
    h = 1e-5
    for trial in range(4):
        n = S.shape[1]
        G = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if np.iscomplexobj(S) else 0)
        G = 0.5 * (G + G.conj().T)
        G /= np.linalg.norm(G)
        D = Lc @ G @ Lc.conj().T
        Gh = rng.standard_normal((M, M)) + (1j * rng.standard_normal((M, M)) if np.iscomplexobj(H) else 0)
        Gh = 0.5 * (Gh + Gh.conj().T)
        Gh /= np.linalg.norm(Gh)
        Ls = O.spinor_overlap(Lc) if spin == "noncollinear" else Lc
        Dh = Ls @ Gh @ Ls.conj().T
        fd_h = (_loss_and_grads(H + h * Dh[None], S, kT, ne, spin, rt, a_eps)[0]
                - _loss_and_grads(H - h * Dh[None], S, kT, ne, spin, rt, a_eps)[0]) / (2 * h)
        fd_s = (_loss_and_grads(H, S + h * D[None], kT, ne, spin, rt, a_eps)[0]
                - _loss_and_grads(H, S - h * D[None], kT, ne, spin, rt, a_eps)[0]) / (2 * h)
        ad_h = float(np.real(np.sum(Hb[0].conj() * Dh)))
        ad_s = float(np.real(np.sum(Sb[0].conj() * D)))
        for fd, ad in ((fd_h, ad_h), (fd_s, ad_s)):
            assert abs(fd - ad) <= 1e-6 * max(abs(fd), abs(ad), 1e-3), (fd, ad)


def test_adjoint_free_energy_identity():
    """F = Omega + mu n_elec with Omega = -kT g_s sum ln(1 + e^{-x}): at fixed n_elec,
    dF/dH = rho and dF/dS = -C diag(g_s f eps) C^H, exactly; the adjoint with explicit
    eigenvalue weights w g_s f must return them."""
    H, S = I.random_pencil(15, 21, True, 20.0)
    kT = 0.1
    r = O.solve(H[None], S[None], kT, 9.0)
    Hb, Sb = O.adjoint(r, kT, eps_bar=2.0 * r.occ)
    assert np.abs(Hb[0] - r.rho[0]).max() <= 1e-12 * np.abs(r.rho[0]).max()
    E = (r.C[0] * (2.0 * r.occ[0] * r.eps[0])[None, :]) @ r.C[0].conj().T
    assert np.abs(Sb[0] + E).max() <= 1e-12 * np.abs(E).max()


# ------------------------------------------------------------------ truth refinement

@pytest.mark.parametrize("cplx", [False, True])
def test_dd_matmul_against_exact_rationals(cplx):
    """The double-double product equals the exact rational product to ~2^-63 of the scales
    (FP64 gets ~2^-53): checked entrywise with fractions on a few entries."""
    from fractions import Fraction
    rng = np.random.default_rng(11 + cplx)
    A = rng.standard_normal((37, 61)) * 10.0 ** rng.uniform(-3, 3, (37, 1))
    B = rng.standard_normal((61, 29)) * 10.0 ** rng.uniform(-3, 3, (1, 29))
    if cplx:
        A = A + 1j * rng.standard_normal(A.shape)
        B = B + 1j * rng.standard_normal(B.shape)
    hi, lo = O.dd_matmul(A, B)
    for (i, j) in [(0, 0), (5, 17), (36, 28), (20, 3)]:
        for part in (np.real, np.imag) if cplx else (np.real,):
            if part is np.real:
                ex = sum(Fraction(float(np.real(A[i, k]))) * Fraction(float(np.real(B[k, j])))
                         - Fraction(float(np.imag(A[i, k]))) * Fraction(float(np.imag(B[k, j]))) for k in range(61))
            else:
                ex = sum(Fraction(float(np.real(A[i, k]))) * Fraction(float(np.imag(B[k, j])))
                         + Fraction(float(np.imag(A[i, k]))) * Fraction(float(np.real(B[k, j]))) for k in range(61))
            got = Fraction(float(part(hi[i, j]))) + Fraction(float(part(lo[i, j])))
            scale = float(np.abs(A[i]).max() * np.abs(B[:, j]).max()) * 61
            assert abs(float(got - ex)) <= 2.0 ** -60 * scale


@pytest.mark.parametrize("n,s", [(40, 0.0), (40, 0.3), (97, -0.2)])
def test_refine_truth_generalized_chain(n, s):
    """Refined eigenvalues of the generalized chain match (e0 + 2t cos th)/(1 + 2s cos th)
    to a few units of the closed form's own rounding, tighter than the FP64 solve."""
    e0, t = 0.2, -0.7
    H = np.diag(np.full(n, e0)) + np.diag(np.full(n - 1, t), 1) + np.diag(np.full(n - 1, t), -1)
    S = np.eye(n) + np.diag(np.full(n - 1, s), 1) + np.diag(np.full(n - 1, s), -1)
    eps, C = O.eigh_generalized(H, S)
    lam, _ = O.refine_truth(H, S, eps, C)
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    ref = np.sort((e0 + 2 * t * np.cos(th)) / (1 + 2 * s * np.cos(th)))
    assert np.abs(np.sort(lam) - ref).max() <= 8 * O.U_ROUND * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [3, 5])
@pytest.mark.parametrize("cplx", [False, True])
def test_refine_truth_exact_roots(n, cplx):
    """On the exact-rational pencils the refined eigenvalues reach the 30-digit roots to
    about the rounding of the stored matrices."""
    sp = pytest.importorskip("sympy")
    Hs, Ss = _rational_pencil(n, 1000 + n + (50 if cplx else 0), cplx)
    lam = sp.Symbol("lam")
    poly = sp.Poly(sp.expand((Hs - lam * Ss).det()), lam)
    coeffs = [sp.re(c) for c in poly.all_coeffs()]
    roots = np.array(sorted(float(r.evalf(30)) for r in sp.Poly(coeffs, lam).real_roots()))
    H = np.array(Hs.evalf(), dtype=complex if cplx else float)
    S = np.array(Ss.evalf(), dtype=complex if cplx else float)
    eps, C = O.eigh_generalized(H, S)
    ref_lam, _ = O.refine_truth(H, S, eps, C)
    beta = O.eig_condition(H, S, eps, C)
    assert np.all(np.abs(np.sort(ref_lam) - roots) <= np.maximum(4 * O.U_ROUND * np.abs(roots), beta))


@pytest.mark.parametrize("tiling", [(1, 1, 1), (2, 1, 1)])
def test_oracle_within_its_bound_of_the_truth(tiling):
    """On the ill-conditioned Si basis the FP64 oracle sits within 8 beta_i of the refined
    eigenvalues of the stored pencil (the gate the GPU path is held to), and the refinement
    has converged (a further sweep moves nothing beyond rounding)."""
    p = I.collinear_gamma(tiling, 0, 0.01)
    H, S = p.H.numpy()[0], p.S.numpy()[0]
    eps, C = O.eigh_generalized(H, S)
    lam, X = O.refine_truth(H, S, eps, C, sweeps=3)
    lam4, _ = O.refine_truth(H, S, eps, C, sweeps=4)
    beta = O.eig_condition(H, S, eps, C)
    assert np.all(np.abs(eps - lam) <= np.maximum(1e-10, 8 * beta))
    assert np.abs(lam4 - lam).max() <= 1e-13 * max(1.0, np.abs(lam).max())


# ------------------------------------------------------------------ two-stage stage references

@pytest.mark.parametrize("cplx", [False, True])
def test_householder_reflector(cplx):
    rng = np.random.default_rng(21 + cplx)
    for m in (1, 2, 7):
        x = rng.standard_normal(m) + (1j * rng.standard_normal(m) if cplx else 0)
        v, tau, beta = O.householder(x)
        H = np.eye(m) - tau * np.outer(v, np.conj(v))
        y = H.conj().T @ x
        assert abs(y[0] - beta) <= 1e-14 * np.linalg.norm(x) and np.abs(y[1:]).max(initial=0.0) <= 1e-14 * np.linalg.norm(x)
        assert np.abs(H.conj().T @ H - np.eye(m)).max() <= 1e-14
    v, tau, beta = O.householder(np.array([2.0, 0.0, 0.0]))  # nothing to annihilate
    assert tau == 0.0 and beta == 2.0


def _chain_in_random_basis(n, cplx, seed):
    """A = Q C Q^H with C the S = I chain (eigenvalues e0 + 2t cos(j pi/(n+1))) and Q a random
    unitary: the closed-form spectrum hidden in a dense Hermitian matrix."""
    rng = np.random.default_rng(seed)
    e0, t = 0.3, -1.0
    C = np.diag(np.full(n, e0)) + np.diag(np.full(n - 1, t), 1) + np.diag(np.full(n - 1, t), -1)
    Z = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Q, _ = np.linalg.qr(Z)
    A = Q @ C @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    lam = np.sort(e0 + 2 * t * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    return A, lam


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(40, 4), (37, 6), (25, 1), (30, 8)])
def test_band_reduce_and_bulge_chase(cplx, n, b):
    """Dense -> band -> tridiagonal: exact zeros outside the band / tridiagonal (to rounding),
    unitary transforms that reproduce their input, and the chain's closed-form spectrum at
    the end (tridiagonal eigenvalues by the oracle's implicit QL after a diagonal phase)."""
    A, lam = _chain_in_random_basis(n, cplx, 100 * n + b + cplx)
    i, j = np.indices((n, n))
    B, Q1 = O.band_reduce(A, b)
    scale = np.abs(A).max()
    if (np.abs(i - j) > b).any():
        assert np.abs(B[np.abs(i - j) > b]).max() <= 1e-13 * scale
    assert np.abs(Q1 @ B @ Q1.conj().T - A).max() <= 1e-13 * scale
    assert np.abs(Q1.conj().T @ Q1 - np.eye(n)).max() <= 1e-13
    T, Q2 = O.bulge_chase(B, b)
    assert np.abs(T[np.abs(i - j) > 1]).max() <= 1e-13 * scale
    assert np.abs(Q2 @ T @ Q2.conj().T - B).max() <= 1e-13 * scale
    assert np.abs(Q2.conj().T @ Q2 - np.eye(n)).max() <= 1e-13
    d = np.real(np.diag(T))
    e = np.abs(np.diag(T, -1))
    ev, _ = O.tridiagonal_eig(d, e)
    assert np.abs(np.sort(ev) - lam).max() <= 1e-13 * n


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b,nbs", [(40, 4, 4), (37, 6, 5), (30, 3, 8), (25, 1, 3)])
def test_bulge_chase_reflectors_regroup_into_blocks(cplx, n, b, nbs):
    """The bulge-chasing reflectors, regrouped into sweep-group x window blocks and applied
    groups-descending / windows-ascending as compact WY blocks, reproduce Q2 X."""
    rng = np.random.default_rng(7 * n + b + cplx)
    Xr = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    B, _ = O.band_reduce(Xr + Xr.conj().T, b)
    refl = []
    _, Q2 = O.bulge_chase(B, b, refl)
    Y = rng.standard_normal((n, 7)) + (1j * rng.standard_normal((n, 7)) if cplx else 0)
    assert np.abs(O.apply_q2_grouped(refl, Y, nbs) - Q2 @ Y).max() <= 1e-13 * np.abs(Y).max()


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,b", [(40, 4), (37, 6), (25, 1), (30, 8), (20, 3), (12, 11)])
def test_band_reduce_panel_form_matches_columnwise(cplx, n, b):
    """The panel form (QR of the block below the band, X = A V T, W = X - V T^H V^H X / 2,
    A22 -= V W^H + W V^H) gives the band of the column-by-column reduction, partial last
    panels included, with a unitary Q1 that reproduces A."""
    rng = np.random.default_rng(3 * n + b + cplx)
    Xr = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    A = Xr + Xr.conj().T
    B1, _ = O.band_reduce(A, b)
    B2, Q = O.band_reduce_blocked(A, b)
    scale = np.abs(A).max()
    assert np.abs(B1 - B2).max() <= 1e-13 * scale
    assert np.abs(Q @ B2 @ Q.conj().T - A).max() <= 1e-13 * scale
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() <= 1e-13


# ------------------------------------------------------------------ conventions and variants

def test_phase_fix_convention():
    """The largest-modulus entry of every column becomes real positive, the lowest row on
    ties; the column changes only by a unit-modulus factor."""
    rng = np.random.default_rng(11)
    C = (rng.standard_normal((9, 5)) + 1j * rng.standard_normal((9, 5))) * 0.1
    C[3, 0] = 2.0 * np.exp(1j * 0.7)                    # unique maximum
    C[2, 1] = 3.0 + 4.0j                                 # exact tie: rows 2 and 6 both modulus 5
    C[6, 1] = -4.0 + 3.0j
    C[:, 2] = 0.0                                        # zero column stays zero
    C[8, 3] = -4.0                                       # negative real maximum
    C[0, 4] = 1j * 3.0
    C[4, 4] = -3.0                                       # tie between rows 0 and 4
    F = O.phase_fix(C)
    expect_row = {0: 3, 1: 2, 3: 8, 4: 0}
    for j, r in expect_row.items():
        assert abs(F[r, j].imag) <= 4 * O.U_ROUND * abs(F[r, j]) and F[r, j].real > 0
        assert np.argmax(np.abs(F[:, j])) == r
        assert abs(abs(F[r, j]) - abs(C[r, j])) <= 1e-15 * abs(C[r, j])
        ph = F[r, j] / C[r, j]
        assert abs(abs(ph) - 1.0) <= 1e-15
        assert np.abs(F[:, j] - ph * C[:, j]).max() <= 1e-15 * np.abs(C[:, j]).max()
    assert np.all(F[:, 2] == 0.0)
    # real columns: the sign makes the largest entry positive
    R = rng.standard_normal((6, 3))
    R[5, 0] = -9.0
    FR = O.phase_fix(R)
    assert FR[5, 0] == 9.0 and np.array_equal(FR[:, 0], -R[:, 0])


def test_hermitian_norm2_power_iteration():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((80, 80)) + 1j * rng.standard_normal((80, 80)))
    lam = np.concatenate([[-7.0, 5.0], rng.uniform(-3, 3, 78)])
    A = (Q * lam) @ Q.conj().T
    assert abs(O.hermitian_norm2(A) - 7.0) <= 1e-6 * 7.0
    assert O.hermitian_norm2(A) <= 7.0 * (1 + 1e-12)


@pytest.mark.parametrize("n,s", [(5, 0.2), (40, -0.3), (90, 0.45)])
def test_lowdin_generalized_chain_closed_form(n, s):
    """The Loewdin route (eig S, V = U s^-1/2, V^H H V, C = V C') on the generalized chain."""
    e0, t = -0.5, 0.7
    H, S = I.chain(n, e0, t, s)
    eps, C = O.eigh_lowdin(H, S)
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    ref = np.sort((e0 + 2 * t * np.cos(th)) / (1 + 2 * s * np.cos(th)))
    assert np.abs(eps - ref).max() <= 1e-12 * max(1, np.abs(ref).max())
    assert np.abs(C.T @ S @ C - np.eye(n)).max() <= 1e-12
    e2, C2 = O.eigh_generalized(H, S)
    assert _match_columns(C, C2) <= 1e-10


@pytest.mark.parametrize("cplx", [False, True])
def test_lowdin_matches_cholesky_route(cplx):
    H, S = I.random_pencil(70, 17, cplx, cond=1e3)
    e1, C1 = O.eigh_lowdin(H, S)
    e2, C2 = O.eigh_generalized(H, S)
    assert np.abs(e1 - e2).max() <= 1e-11 * np.abs(e2).max()
    assert _match_columns(C1, C2) <= 1e-8


def test_spin_polarized_identical_channels_reduce_to_collinear():
    """Equal up and down channels: each carries the collinear spectrum, mu is the collinear
    one, rho_up + rho_down is the collinear rho (g_s = 2 split into two g_s = 1 channels)."""
    p = I.collinear_gamma((1, 1, 1), 0, 0.01)
    H, S = p.H.numpy(), p.S.numpy()
    col = O.solve(H, S, p.kT, p.n_elec)
    Hs = np.stack([H, H], axis=1)
    sp = O.solve(Hs, S, p.kT, p.n_elec, spin="spin_polarized")
    assert np.array_equal(sp.eps[0, 0], col.eps[0]) and np.array_equal(sp.eps[0, 1], col.eps[0])
    assert abs(sp.mu - col.mu) <= 1e-12
    assert np.abs(sp.rho[0, 0] + sp.rho[0, 1] - col.rho[0]).max() <= 1e-9 * np.abs(col.rho[0]).max()
    assert abs(sp.e_band - col.e_band) <= 1e-10 * abs(col.e_band)


def test_spin_polarized_uniform_exchange_shifts_spectra():
    """H_up/down = H -/+ D S (a uniform S-consistent exchange shift): the channels' spectra
    are the collinear one shifted by -D and +D exactly."""
    H, S = I.random_pencil(40, 23, False, cond=1e2)
    D = 0.05
    Hs = np.stack([H - D * S, H + D * S])[None]
    sp = O.solve(Hs, S[None], 0.05, 30.0, spin="spin_polarized")
    e, _ = O.eigh_generalized(H, S)
    assert np.abs(sp.eps[0, 0] - (e - D)).max() <= 1e-12 * np.abs(e).max()
    assert np.abs(sp.eps[0, 1] - (e + D)).max() <= 1e-12 * np.abs(e).max()
    # both channels share one mu: total electrons = n_elec, g_s = 1
    tr = sum(np.trace(sp.rho[0, s_] @ S) for s_ in range(2))
    assert abs(tr - 30.0) <= 1e-10 * 30.0


def test_energy_density_matrix_chain_closed_form():
    """S = I chain: E = C diag(g_s f eps) C^T with the sine eigenvectors and cosine
    eigenvalues of the closed form; tr(E S) = sum g_s f eps."""
    n, e0, t, kT = 30, 0.3, -1.0, 0.05
    H, S = I.chain(n, e0, t)
    res = O.solve(H[None], S[None], kT, 22.0)
    j = np.arange(1, n + 1)
    eps = e0 + 2 * t * np.cos(j * np.pi / (n + 1))
    V = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * np.pi / (n + 1))
    f = O.fermi((eps - res.mu) / kT)
    ref = (V * (2.0 * f * eps)[None, :]) @ V.T
    E = O.energy_density_matrix(res.C[0], res.occ[0], res.eps[0], 2.0)
    assert np.abs(E - ref).max() <= 1e-12
    assert abs(np.trace(E @ S) - np.sum(2.0 * f * eps)) <= 1e-12 * n
