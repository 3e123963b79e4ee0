"""CPU oracle for the generalized Kohn-Sham eigensolve and density matrix.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's
CPU-baseline leg.  The product path never imports this module and shares no code with
it.  Everything here is plain FP64:

* the eigensolve (paper Sec. 2, H C = S C eps; Sec. 2 Bloch form per k; Sec. 2/3.2
  noncollinear spinor with S_NC = I_2 (x) S) runs in the unblocked C code of
  gks_oracle.c (Cholesky, explicit substitution, Householder, implicit QL, back
  substitution);
* occupations, chemical potential, band energy and density matrix (paper Sec. 3.1
  Parts 3 and 4; Sec. 2 density-matrix definition) are direct numpy sums;
* refine_truth: Ogita-Aishima refinement of those eigenpairs with double-double residual
  products, a reference beyond the FP64 rounding of the eigensolver itself;
* band_reduce / bulge_chase: stage references for a two-stage tridiagonalization.

Readings where the paper is silent (each listed in the design notes):
* Fermi-Dirac f(x) = 1/(1+e^x), x = (eps - mu)/kT (the paper names f_i only);
* spin factor g_s = 2 collinear, 1 noncollinear (Sec. 2 electron density, with and
  without the factor 2);
* mu by bisection on the increasing electron count, shared by all k of a system,
  weights w_k (default 1/nk); bracket [min eps - 1, max eps + 1], stop when
  hi - lo <= 4u max(1, |mu|) or after 200 halvings;
* rho_k = C_k diag(g_s f_k) C_k^H over the columns with f >= f_cut = 1e-16.  The paper's
  n_lm = sum_i f_i c*_li c_mi is conj(rho)/g_s, i.e. its transpose for Hermitian rho.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgks_oracle.so")
_lib = None

F_CUT = 1e-16
U_ROUND = 2.0 ** -53


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc with OpenMP, no architecture-specific flags)."""
    src = os.path.join(_HERE, "gks_oracle.c")
    inc = os.path.join(_HERE, "oracle_core.inc")
    newest = max(os.path.getmtime(src), os.path.getmtime(inc))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        for sfx in ("d", "z"):
            getattr(lib, f"oracle_solve_{sfx}").argtypes = [ctypes.c_int, P, P, P, P]
            getattr(lib, f"oracle_chol_{sfx}").argtypes = [ctypes.c_int, P]
            getattr(lib, f"oracle_reduce_{sfx}").argtypes = [ctypes.c_int, P, P]
            getattr(lib, f"oracle_tridiag_{sfx}").argtypes = [ctypes.c_int, P, P, P, P, P]
            getattr(lib, f"oracle_backtransform_{sfx}").argtypes = [ctypes.c_int, P, P, P, P, P]
            getattr(lib, f"oracle_unreduce_{sfx}").argtypes = [ctypes.c_int, P, P]
            getattr(lib, f"oracle_unreduce_{sfx}").restype = None
            getattr(lib, f"oracle_reduce_{sfx}").restype = None
            getattr(lib, f"oracle_tridiag_{sfx}").restype = None
            getattr(lib, f"oracle_backtransform_{sfx}").restype = None
        lib.oracle_tridiag_eig.argtypes = [ctypes.c_int, P, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _sfx(a):
    return "z" if np.iscomplexobj(a) else "d"


class OracleError(RuntimeError):
    pass


# ----------------------------- single-pencil stages -----------------------------

def cholesky(S: np.ndarray) -> np.ndarray:
    """Step 1: S = L L^H (lower triangle of S read)."""
    L = np.array(S, dtype=S.dtype, order="C", copy=True)
    rc = getattr(_load(), f"oracle_chol_{_sfx(L)}")(L.shape[0], _ptr(L))
    if rc:
        raise OracleError(f"S not positive definite at column {rc - 1}")
    return L


def reduce_standard(L: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Step 2: H' = L^-1 H L^-H."""
    A = np.array(H, dtype=L.dtype, order="C", copy=True)
    getattr(_load(), f"oracle_reduce_{_sfx(A)}")(A.shape[0], _ptr(np.ascontiguousarray(L)), _ptr(A))
    return A


def tridiagonalize(A: np.ndarray):
    """Step 3: Householder reduction. Returns (d, sub, U, beta)."""
    A = np.array(A, order="C", copy=True)
    n = A.shape[0]
    d = np.zeros(n)
    sub = np.zeros(max(n - 1, 1), dtype=A.dtype)
    U = np.zeros((n, n), dtype=A.dtype)
    beta = np.zeros(n)
    getattr(_load(), f"oracle_tridiag_{_sfx(A)}")(n, _ptr(A), _ptr(d), _ptr(sub), _ptr(U), _ptr(beta))
    return d, sub[: max(n - 1, 0)], U, beta


# ----------------------------- two-stage reduction (stage references) -----------------------------
#
# Dense -> band -> tridiagonal, written as plain full-matrix Householder similarity
# transforms so that every step can be read against its definition.  Stage references for
# a two-stage tridiagonalization (the scope's dense-to-band and band-to-tridiagonal rows);
# the one-stage oracle above remains the reference for the full eigensolve.

def householder(x: np.ndarray):
    """(v, tau, beta) with v[0] = 1 and (I - tau v v^H)^H x = beta e_1, beta real."""
    x = np.asarray(x)
    alpha = x[0]
    xn = np.linalg.norm(x[1:]) if x.size > 1 else 0.0
    v = np.zeros_like(x)
    v[0] = 1.0
    if xn == 0.0 and np.imag(alpha) == 0.0:
        return v, 0.0 * alpha, np.real(alpha)
    beta = -np.copysign(np.sqrt(np.abs(alpha) ** 2 + xn ** 2), np.real(alpha))
    tau = (beta - alpha) / beta
    v[1:] = x[1:] / (alpha - beta)
    return v, tau, beta


def _apply_similarity(A, Q, v, tau, r0):
    """A <- H^H A H, Q <- Q H with H = I - tau v v^H acting on rows/columns r0.."""
    n = A.shape[0]
    H = np.eye(n, dtype=A.dtype)
    k = v.size
    H[r0:r0 + k, r0:r0 + k] -= tau * np.outer(v, np.conj(v))
    return H.conj().T @ A @ H, Q @ H


def band_reduce(A: np.ndarray, b: int):
    """Hermitian A -> (B, Q1) with A = Q1 B Q1^H and B banded: B_ij = 0 for |i - j| > b.
    Column j's entries below row j + b are annihilated by a reflector on rows j + b.."""
    A = np.array(A, dtype=np.result_type(A, np.float64), copy=True)
    n = A.shape[0]
    Q = np.eye(n, dtype=A.dtype)
    for j in range(n - b - 1):
        v, tau, _ = householder(A[j + b:, j])
        A, Q = _apply_similarity(A, Q, v, tau, j + b)
    return A, Q


def band_reduce_blocked(A: np.ndarray, b: int):
    """The same dense -> band reduction in panel form: for the panel of columns [k, k+b),
    QR of the block below the band by Householder reflectors (V unit lower trapezoidal,
    T from the forward accumulation), then the two-sided update of the trailing block
        X = A22 V T,  W = X - (1/2) V (T^H V^H X),  A22 <- A22 - V W^H - W V^H.
    Returns (B, Q1) like band_reduce (same reflectors, so the same B up to rounding)."""
    A = np.array(A, dtype=np.result_type(A, np.float64), copy=True)
    n = A.shape[0]
    Q = np.eye(n, dtype=A.dtype)
    for k in range(0, max(n - b - 1, 0), b):
        r0 = k + b               # first row below the band for this panel
        kb = min(b, n - b - 1 - k)  # columns of the panel that still have entries to annihilate
        m = n - r0
        P = A[r0:, k:k + b].copy()  # all b columns of the panel receive Q^H; kb reflectors
        V = np.zeros((m, kb), dtype=A.dtype)
        taus = np.zeros(kb, dtype=A.dtype)
        for c in range(kb):      # unblocked QR of the panel
            v, tau, _ = householder(P[c:, c])
            V[c:, c] = v
            taus[c] = tau
            P[c:, c:] -= np.outer(v, (np.conj(tau) * (np.conj(v) @ P[c:, c:])))
        Tm = np.zeros((kb, kb), dtype=A.dtype)
        for c in range(kb):
            Tm[:c, c] = -taus[c] * (Tm[:c, :c] @ (V[:, :c].conj().T @ V[:, c]))
            Tm[c, c] = taus[c]
        # panel and its mirror: Q^H applied from the left to the panel columns
        A[r0:, k:k + b] = P
        A[k:k + b, r0:] = P.conj().T
        A22 = A[r0:, r0:]
        X = A22 @ V @ Tm
        W = X - 0.5 * V @ (Tm.conj().T @ (V.conj().T @ X))
        A[r0:, r0:] = A22 - V @ W.conj().T - W @ V.conj().T
        Q[:, r0:] = Q[:, r0:] - (Q[:, r0:] @ V) @ Tm @ V.conj().T
    return A, Q


def bulge_chase(B: np.ndarray, b: int, reflectors: list | None = None):
    """Banded Hermitian B (bandwidth b) -> (T, Q2) with B = Q2 T Q2^H, T tridiagonal.
    Sweep i annihilates column i below the subdiagonal with a reflector on rows i+1..i+b;
    the fill it creates below the band is chased down: the reflector of the next window
    (rows r0..r0+b-1, r0 one past the previous window) annihilates the first column of
    the previous window below row r0, until the window leaves the matrix.  Window j of
    sweep i starts at row i + 1 + j b.  With `reflectors` (a list), each reflector is
    appended as (i, j, first row, v, tau) in generation order, Q2 = their product."""
    T = np.array(B, dtype=np.result_type(B, np.float64), copy=True)
    n = T.shape[0]
    Q = np.eye(n, dtype=T.dtype)
    for i in range(n - 2):
        r0, r1 = i + 1, min(i + b, n - 1)
        v, tau, _ = householder(T[r0:r1 + 1, i])
        T, Q = _apply_similarity(T, Q, v, tau, r0)
        if reflectors is not None:
            reflectors.append((i, 0, r0, v, tau))
        c, j = r0, 0
        while True:
            q0 = r1 + 1
            if q0 >= n:
                break
            q1 = min(q0 + b - 1, n - 1)
            v, tau, _ = householder(T[q0:q1 + 1, c])
            T, Q = _apply_similarity(T, Q, v, tau, q0)
            j += 1
            if reflectors is not None:
                reflectors.append((i, j, q0, v, tau))
            c, r1 = q0, q1
    return T, Q


def apply_q2_grouped(reflectors: list, X: np.ndarray, nbs: int) -> np.ndarray:
    """Q2 X with the bulge-chasing reflectors regrouped for block application: sweeps in
    groups of nbs, and within a group one block per window index j,
    B_{g,j} = H_{s0,j} H_{s0+1,j} ... (compact WY, I - V T V^H).  Since a reflector of sweep
    s, window j meets none of later sweeps' higher windows, Q2 = prod_g prod_{j desc}
    B_{g,j}; so X is multiplied by groups from the last, windows ascending."""
    X = np.array(X, dtype=np.result_type(X, reflectors[0][3] if reflectors else X), copy=True)
    groups = {}
    for (i, j, r0, v, tau) in reflectors:
        groups.setdefault(i // nbs, {}).setdefault(j, []).append((r0, v, tau))
    for g in sorted(groups, reverse=True):
        for j in sorted(groups[g]):
            blk = groups[g][j]  # sweeps ascending
            top = min(r0 for r0, _, _ in blk)
            bot = max(r0 + v.size for r0, v, _ in blk)
            k = len(blk)
            V = np.zeros((bot - top, k), dtype=X.dtype)
            for c, (r0, v, _) in enumerate(blk):
                V[r0 - top:r0 - top + v.size, c] = v
            taus = [t for _, _, t in blk]
            Tm = np.zeros((k, k), dtype=X.dtype)
            for c in range(k):  # forward accumulation: T[:c, c] = -tau_c T[:c,:c] V[:, :c]^H v_c
                Tm[:c, c] = -taus[c] * (Tm[:c, :c] @ (V[:, :c].conj().T @ V[:, c]))
                Tm[c, c] = taus[c]
            X[top:bot] -= V @ (Tm @ (V.conj().T @ X[top:bot]))
    return X


def tridiagonal_eig(d: np.ndarray, e: np.ndarray):
    """Step 4-5: implicit QL on the real tridiagonal; ascending eigenvalues, vectors Z."""
    n = d.shape[0]
    dd = np.array(d, dtype=np.float64, copy=True)
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = e
    Z = np.eye(n)
    rc = _load().oracle_tridiag_eig(n, _ptr(dd), _ptr(ee), _ptr(Z))
    if rc:
        raise OracleError(f"implicit QL did not converge (block at {rc - 1})")
    return dd, Z


def back_transform(sub, U, beta, Z):
    """Step 6a: X = Q D Z."""
    n = Z.shape[0]
    X = np.zeros((n, n), dtype=U.dtype)
    s = np.zeros(max(n, 1), dtype=U.dtype)
    s[: n - 1] = sub
    getattr(_load(), f"oracle_backtransform_{_sfx(U)}")(n, _ptr(s), _ptr(U), _ptr(beta),
                                                        _ptr(np.ascontiguousarray(Z)), _ptr(X))
    return X


def unreduce(L, X):
    """Step 6b: C = L^-H X."""
    C = np.array(X, order="C", copy=True)
    getattr(_load(), f"oracle_unreduce_{_sfx(C)}")(C.shape[0], _ptr(np.ascontiguousarray(L)), _ptr(C))
    return C


def eigh_generalized(H: np.ndarray, S: np.ndarray):
    """All eigenpairs of one Hermitian pencil (H, S): eps ascending, C with C^H S C = I."""
    cplx = np.iscomplexobj(H) or np.iscomplexobj(S)
    dt = np.complex128 if cplx else np.float64
    H = np.ascontiguousarray(H, dtype=dt)
    S = np.ascontiguousarray(S, dtype=dt)
    n = H.shape[0]
    eps = np.zeros(n)
    C = np.zeros((n, n), dtype=dt)
    rc = getattr(_load(), f"oracle_solve_{_sfx(H)}")(n, _ptr(H), _ptr(S), _ptr(eps), _ptr(C))
    if rc < 0:
        raise OracleError(f"S not positive definite at column {-rc - 1}")
    if rc > 0:
        raise OracleError("implicit QL did not converge")
    return eps, phase_fix(C)


def eigh_lowdin(H: np.ndarray, S: np.ndarray):
    """All eigenpairs of (H, S) by the Loewdin route of the paper (Sec. 3.1 Parts 2-1 to 2-5):
    S = U diag(s) U^H (this oracle's eigensolver on the standard problem S), V = U s^-1/2,
    H' = V^H H V, H' = C' diag(eps) C'^H, C = V C'.  Same eps and C (up to phases within
    degenerate sets) as eigh_generalized in exact arithmetic."""
    cplx = np.iscomplexobj(H) or np.iscomplexobj(S)
    dt = np.complex128 if cplx else np.float64
    S = np.asarray(S, dtype=dt)
    I = np.eye(S.shape[0], dtype=dt)
    s, U = eigh_generalized(S, I)
    if np.any(s <= 0.0):
        raise OracleError("S not positive definite (Loewdin)")
    V = U / np.sqrt(s)[None, :]
    Hp = V.conj().T @ np.asarray(H, dtype=dt) @ V
    Hp = 0.5 * (Hp + Hp.conj().T)
    eps, Cp = eigh_generalized(Hp, I)
    return eps, phase_fix(V @ Cp)


def phase_fix(C: np.ndarray) -> np.ndarray:
    """Column phase convention: the largest-modulus entry (lowest index on ties) is real
    and positive."""
    C = np.array(C, copy=True)
    idx = np.argmax(np.abs(C), axis=0)
    piv = C[idx, np.arange(C.shape[1])]
    mag = np.abs(piv)
    ph = np.where(mag > 0, piv / np.where(mag > 0, mag, 1), 1)
    return C / ph[None, :]


# ----------------------------- occupations and density -----------------------------

def fermi(x: np.ndarray) -> np.ndarray:
    """f(x) = 1/(1+e^x), written so that exp never overflows."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x > 0
    ex = np.exp(-x[pos])
    out[pos] = ex / (1.0 + ex)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def electron_count(mu, eps, w, gs, kT):
    return float(sum(w[k] * gs * fermi((eps[k] - mu) / kT).sum() for k in range(eps.shape[0])))


def chemical_potential(eps: np.ndarray, w: np.ndarray, gs: float, kT: float, n_elec: float):
    """Bisection on N(mu) = sum_k w_k g_s sum_i f((eps_ik - mu)/kT) = n_elec."""
    M = eps.shape[1]
    if not (kT > 0):
        raise OracleError("kT must be positive")
    if not (0.0 < n_elec < gs * M * float(np.sum(w))):
        raise OracleError("n_elec out of range")
    lo = float(eps.min()) - 1.0
    hi = float(eps.max()) + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if hi - lo <= 4.0 * U_ROUND * max(1.0, abs(mid)):
            break
        if electron_count(mid, eps, w, gs, kT) < n_elec:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def density_matrix(C: np.ndarray, occ: np.ndarray, gs: float, f_cut: float = F_CUT):
    """rho = C diag(g_s f) C^H over the columns with f >= f_cut (direct weighted sum)."""
    keep = occ >= f_cut
    Ck = C[:, keep]
    return (Ck * (gs * occ[keep])[None, :]) @ Ck.conj().T


def energy_density_matrix(C: np.ndarray, occ: np.ndarray, eps: np.ndarray, gs: float, f_cut: float = F_CUT):
    """E = C diag(g_s f eps) C^H over the columns with f >= f_cut: the energy-density matrix
    that accompanies rho (paper Sec. 3.1 Part 4, needed for forces); tr(E S) = E_band per k
    before the k weight."""
    keep = occ >= f_cut
    Ck = C[:, keep]
    return (Ck * (gs * occ[keep] * eps[keep])[None, :]) @ Ck.conj().T


@dataclass
class Result:
    eps: np.ndarray        # (nk, M)
    C: np.ndarray          # (nk, M, M)
    mu: float
    occ: np.ndarray        # (nk, M)
    rho: np.ndarray        # (nk, M, M)
    e_band: float
    n_rho: np.ndarray      # (nk,) columns kept in rho


def spinor_overlap(S: np.ndarray) -> np.ndarray:
    """S_NC = diag(S, S) (paper Sec. 3.2)."""
    n = S.shape[0]
    out = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    out[:n, :n] = S
    out[n:, n:] = S
    return out


def solve(H, S, kT: float, n_elec: float, spin: str = "collinear", kweights=None,
          f_cut: float = F_CUT, reduction: str = "cholesky") -> Result:
    """Full path for nk pencils sharing one chemical potential.

    H: (nk, M, M); S: (nk, N, N) with M = N (collinear) or 2N (noncollinear)."""
    H = np.asarray(H)
    S = np.asarray(S)
    if spin == "spin_polarized":
        return _solve_spin_polarized(H, S, kT, n_elec, kweights, f_cut)
    if H.ndim == 2:
        H = H[None]
        S = S[None]
    nk, M = H.shape[0], H.shape[1]
    gs = 2.0 if spin == "collinear" else 1.0
    w = np.full(nk, 1.0 / nk) if kweights is None else np.asarray(kweights, float)
    eps = np.zeros((nk, M))
    dt = np.complex128 if (np.iscomplexobj(H) or np.iscomplexobj(S) or spin != "collinear") else np.float64
    C = np.zeros((nk, M, M), dtype=dt)
    eig = eigh_lowdin if reduction == "lowdin" else eigh_generalized
    for k in range(nk):
        Sk = spinor_overlap(S[k]) if spin == "noncollinear" else S[k]
        eps[k], C[k] = eig(H[k].astype(dt), Sk.astype(dt))
    mu = chemical_potential(eps, w, gs, kT, n_elec)
    occ = np.stack([fermi((eps[k] - mu) / kT) for k in range(nk)])
    rho = np.stack([density_matrix(C[k], occ[k], gs, f_cut) for k in range(nk)])
    e_band = float(sum(w[k] * gs * np.sum(occ[k] * eps[k]) for k in range(nk)))
    n_rho = np.array([int(np.sum(occ[k] >= f_cut)) for k in range(nk)])
    return Result(eps, C, mu, occ, rho, e_band, n_rho)


def _solve_spin_polarized(H, S, kT, n_elec, kweights, f_cut):
    """Spin-polarized collinear run (paper Sec. 2, one Kohn-Sham problem per spin channel):
    H (nk, 2, N, N) holds the up and down channels of each k-point, S (nk, N, N) is shared by
    both.  Each channel is solved on its own; one mu for all k-points and both channels,
    g_s = 1, the weight w_k applying to both channels.  Arrays keep the channel axis after k."""
    if H.ndim == 3:
        H = H[None]
        S = S[None]
    nk, _, N, _ = H.shape
    w = np.full(nk, 1.0 / nk) if kweights is None else np.asarray(kweights, float)
    dt = np.complex128 if (np.iscomplexobj(H) or np.iscomplexobj(S)) else np.float64
    eps = np.zeros((nk, 2, N))
    C = np.zeros((nk, 2, N, N), dtype=dt)
    for k in range(nk):
        for s_ in range(2):
            eps[k, s_], C[k, s_] = eigh_generalized(H[k, s_].astype(dt), S[k].astype(dt))
    flat = eps.reshape(2 * nk, N)
    wi = np.repeat(w, 2)
    mu = chemical_potential(flat, wi, 1.0, kT, n_elec)
    occ = np.stack([fermi((flat[i] - mu) / kT) for i in range(2 * nk)]).reshape(nk, 2, N)
    rho = np.stack([[density_matrix(C[k, s_], occ[k, s_], 1.0, f_cut) for s_ in range(2)] for k in range(nk)])
    e_band = float(sum(w[k] * np.sum(occ[k] * eps[k]) for k in range(nk)))
    n_rho = np.array([[int(np.sum(occ[k, s_] >= f_cut)) for s_ in range(2)] for k in range(nk)])
    return Result(eps, C, mu, occ, rho, e_band, n_rho)


# ----------------------------- error measures -----------------------------

def hermitian_norm2(A, iters: int = 300, seed: int = 0) -> float:
    """||A||_2 of a Hermitian A by power iteration (the largest |eigenvalue|): a lower bound
    that reaches the norm to well under a percent after a few hundred steps; O(iters n^2),
    for orders where a full SVD would dominate the oracle's own cost."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(A.shape[0]).astype(A.dtype)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = A @ v
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
    return lam


def eig_condition(H, S, eps, C, norms=None):
    """beta_i = u (||H||_2 + |eps_i| ||S||_2) ||c_i||_2^2: first-order FP64 floor of eps_i
    for a backward-stable method on an S-normalized eigenpair.  norms = (||H||_2, ||S||_2)
    if already known (e.g. from hermitian_norm2 at large orders)."""
    nh, ns = norms if norms is not None else (np.linalg.norm(H, 2), np.linalg.norm(S, 2))
    cn = np.sum(np.abs(C) ** 2, axis=0)
    return U_ROUND * (nh + np.abs(eps) * ns) * cn


# ----------------------------- truth refinement -----------------------------
#
# A reference beyond FP64 rounding of the computation: Ogita-Aishima refinement steps
# (Ogita & Aishima 2018, generalized here with the S inner product) applied to the
# oracle's eigenpairs of the stored FP64 pencil, with the residual products X^H S X and
# X^H H X evaluated to about twice FP64 precision.  Those products use error-free
# splitting (Ozaki, Ogita, Oishi, Rump): every entry is cut into three 21-bit slices
# relative to its row's (or column's) largest entry, each slice product is then an exact
# FP64 matrix product (21 + 21 bits per term, at most 2^11 terms), and the slice products
# are summed in double-double arithmetic (Knuth's TwoSum).

def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _slices(X, axis, nbits=21, count=3):
    """Real X = 2^e (sum_s D_s 2^{-nbits (s+1)}) + remainder below 2^{e - nbits count},
    e per row (axis=1) or column (axis=0); D_s integer-valued."""
    m = np.max(np.abs(X), axis=axis, keepdims=True)
    e = np.where(m > 0, np.ceil(np.log2(np.where(m > 0, m, 1.0))) + 1, 0.0)
    r = np.ldexp(X, (-e).astype(int))
    out = []
    for _ in range(count):
        t = np.ldexp(r, nbits)
        d = np.trunc(t)
        out.append(d)
        r = t - d
    return e, out


def _dd_matmul_real(A, B, nbits=21, count=3):
    """(hi, lo) with hi + lo = A @ B to about 2^-(nbits count) of the row and column scales."""
    if A.shape[1] > 2 ** (53 - 2 * nbits):
        raise ValueError("inner dimension too large for exact slice products")
    ea, As = _slices(A, 1, nbits, count)
    eb, Bs = _slices(B, 0, nbits, count)
    hi = np.zeros((A.shape[0], B.shape[1]))
    lo = np.zeros_like(hi)
    for s in range(count):
        for t in range(count):
            if s + t > count:  # below the kept precision
                continue
            P = As[s] @ Bs[t]  # exact: integers below 2^53
            P = np.ldexp(P, (ea + eb - nbits * (s + t + 2)).astype(int))
            hi, err = _two_sum(hi, P)
            lo += err
    return _two_sum(hi, lo)


def dd_matmul(A, B):
    """A @ B (real or complex) as a double-double pair (hi, lo)."""
    if not (np.iscomplexobj(A) or np.iscomplexobj(B)):
        return _dd_matmul_real(np.asarray(A, float), np.asarray(B, float))
    Ar, Ai = np.real(A).astype(float), np.imag(A).astype(float)
    Br, Bi = np.real(B).astype(float), np.imag(B).astype(float)
    parts = []
    for X, Y, sign in ((Ar, Br, 1), (Ai, Bi, -1), (Ar, Bi, 1), (Ai, Br, 1)):
        h, l = _dd_matmul_real(X, Y)
        parts.append((sign * h, sign * l))
    rh, rl = _two_sum(parts[0][0], parts[1][0])
    rl = rl + parts[0][1] + parts[1][1]
    ih, il = _two_sum(parts[2][0], parts[3][0])
    il = il + parts[2][1] + parts[3][1]
    return rh + 1j * ih, rl + 1j * il


def refine_truth(H, S, eps, C, sweeps: int = 3):
    """Refined eigenpairs of the stored pencil (H, S): Ogita-Aishima steps with
    R = I - X^H S X and T = X^H H X in double-double,
        lambda_i = t_ii / (1 - r_ii),  e_ii = r_ii / 2,
        e_ij = (t_ij + lambda_j r_ij) / (lambda_j - lambda_i)  (separated pairs),
        e_ij = r_ij / 2                                         (|lambda_i - lambda_j| <= omega),
        X <- X + X E,
    omega = 2 (||T - diag(lambda)||_2 + ||H||_2 ||R||_2) as in the published method.
    Returns (lambda, X) after `sweeps` steps; lambda carries the double-double residuals'
    accuracy (not FP64 rounding of the eigensolver)."""
    X = np.array(C, dtype=np.result_type(C, H, S))
    nh = np.linalg.norm(H, 2)
    lam = np.asarray(eps, float).copy()
    M = X.shape[1]
    for _ in range(sweeps):
        SXh, SXl = dd_matmul(S, X)
        HXh, HXl = dd_matmul(H, X)
        Xh = X.conj().T
        Gh, Gl = dd_matmul(Xh, SXh)
        Gl = Gl + Xh @ SXl
        Th, Tl = dd_matmul(Xh, HXh)
        Tl = Tl + Xh @ HXl
        R = -(Gh - np.eye(M)) - Gl
        T = Th + Tl
        lam = np.real(np.diag(T)) / (1.0 - np.real(np.diag(R)))
        omega = 2.0 * (np.linalg.norm(T - np.diag(lam), 2) + nh * np.linalg.norm(R, 2))
        D = lam[None, :] - lam[:, None]  # D_ij = lambda_j - lambda_i
        sep = np.abs(D) > omega
        E = np.where(sep, (T + lam[None, :] * R) / np.where(sep, D, 1.0), R / 2.0)
        np.fill_diagonal(E, np.real(np.diag(R)) / 2.0)
        X = X + X @ E
    return lam, X


# ----------------------------- adjoint (vector-Jacobian product) -----------------------------

def fermi_prime(eps, mu, kT):
    """df/d eps = -f (1 - f) / kT."""
    f = fermi((eps - mu) / kT)
    return -f * (1.0 - f) / kT


def adjoint(res: Result, kT: float, spin: str = "collinear", kweights=None, rho_bar=None, eps_bar=None,
            e_band_bar: float = 0.0):
    """Gradients of L(rho, eps, E_band) with respect to H and S (Hermitian), n_elec fixed.

    First-order perturbation of H C = S C eps with C^H S C = I: for M = C^H dH C and
    N = C^H dS C, d eps_i = M_ii - eps_i N_ii and, at fixed mu,
        d rho = g_s C [G o M - G' o N] C^H,
        G_ij  = (f_i - f_j)/(eps_i - eps_j)              (f'_i when eps_i = eps_j),
        G'_ij = (f_i eps_i - f_j eps_j)/(eps_i - eps_j)  (f_i + eps_i f'_i when equal).
    The electron count fixes d mu = sum w f' d eps / sum w f'.  Collecting the terms with
    W = C^H rho_bar C (rho_bar made Hermitian):
        H_bar = C [g_s G o W + diag(e)] C^H,   S_bar = -C [g_s G' o W + diag(eps e)] C^H,
        e_i = eps_bar_i + E_bar g_s w (f_i + eps_i f'_i) + A w f'_i / sum w f',
        A = -g_s sum_k sum_i f'_ki Re W_k,ii - E_bar g_s sum_k w_k sum_i f'_ki eps_ki.
    Noncollinear: S_NC = diag(S, S), so S_bar is the sum of the two diagonal spin blocks.
    Returns (H_bar (nk, M, M), S_bar (nk, N, N))."""
    eps, C, mu = res.eps, res.C, res.mu
    nk, M = eps.shape
    gs = 2.0 if spin == "collinear" else 1.0
    w = np.full(nk, 1.0 / nk) if kweights is None else np.asarray(kweights, float)
    f = np.stack([fermi((eps[k] - mu) / kT) for k in range(nk)])
    fp = np.stack([fermi_prime(eps[k], mu, kT) for k in range(nk)])
    Ws = []
    for k in range(nk):
        if rho_bar is None:
            Ws.append(np.zeros((M, M), dtype=C.dtype))
        else:
            rb = 0.5 * (rho_bar[k] + rho_bar[k].conj().T)
            Ws.append(C[k].conj().T @ rb @ C[k])
    wfp = sum(w[k] * fp[k].sum() for k in range(nk))
    A = -gs * sum(np.sum(fp[k] * Ws[k].diagonal().real) for k in range(nk))
    A -= e_band_bar * gs * sum(w[k] * np.sum(fp[k] * eps[k]) for k in range(nk))
    Hb, Sb = [], []
    for k in range(nk):
        e = np.zeros(M) if eps_bar is None else np.array(eps_bar[k], float)
        e = e + e_band_bar * gs * w[k] * (f[k] + eps[k] * fp[k])
        if wfp != 0.0:
            e = e + A * w[k] * fp[k] / wfp
        d = eps[k][:, None] - eps[k][None, :]
        close = np.abs(d) <= 1e-12 * np.maximum(1.0, np.abs(eps[k]))[:, None]
        dsafe = np.where(close, 1.0, d)
        G = np.where(close, fp[k][:, None], (f[k][:, None] - f[k][None, :]) / dsafe)
        fe = f[k] * eps[k]
        Gp = np.where(close, (f[k] + eps[k] * fp[k])[:, None], (fe[:, None] - fe[None, :]) / dsafe)
        BH = gs * G * Ws[k] + np.diag(e)
        BS = -(gs * Gp * Ws[k] + np.diag(eps[k] * e))
        hb = C[k] @ BH @ C[k].conj().T
        sb = C[k] @ BS @ C[k].conj().T
        Hb.append(0.5 * (hb + hb.conj().T))
        sb = 0.5 * (sb + sb.conj().T)
        if spin == "noncollinear":
            n = M // 2
            sb = sb[:n, :n] + sb[n:, n:]
        Sb.append(sb)
    return np.stack(Hb), np.stack(Sb)
