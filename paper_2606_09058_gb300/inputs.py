"""Seeded synthetic workloads for the generalized Kohn-Sham eigenproblem.

This module builds inputs only: overlap S, Hamiltonian H (collinear, Bloch-summed or
noncollinear spinor) and closed-form test matrices.  It holds none of the solver's
arithmetic and is the one module that both the CPU oracle tests and the CUDA path use.

Physical setting (paper Sec. 4): silicon in the diamond structure (a = 5.431 A =
10.26 bohr), 13 basis functions per atom, a 2x2x2 Monkhorst-Pack k mesh.  The paper's
OpenMX pseudo-atomic orbitals are replaced by 13 normalized s-type Gaussians per atom,
exponents log-spaced 0.1 .. 4.0 bohr^-2, so that N = 13 * atoms as in the paper.

Matrix elements (closed forms for s-Gaussians, p = a+b, mu = ab/p, d = |A-B|):
  S_ab = N_a N_b (pi/p)^{3/2} exp(-mu d^2)                       (overlap, Sec. 2 S_lm)
  T_ab = mu (3 - 2 mu d^2) S_ab                                   (kinetic)
  V    = -Z sum_C |w_C><w_C|,  w_C(r) = exp(-|r-R_C|^2), Z = 4     (per-atom well)
  H    = T + V + 1e-3 * S U S,  U = (A + A^T)/2, A ~ U(-1,1)
The well is taken in separable form and the random term is sandwiched by S so that
H stays bounded relative to S on the near-null space of the overcomplete basis (an
entrywise perturbation of H produces spurious eigenvalues of order 1e7 Ha).

Random draws use numpy PCG64 with seed 9058000 + workload index, in a fixed order.
Heavy dense products run through torch on the requested device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

A_BOHR = 10.26            # diamond Si lattice constant, 5.431 A (paper Sec. 4)
N_PER_ATOM = 13           # s2p2d1 basis size per atom (paper Sec. 4)
EXPONENTS = np.geomspace(0.1, 4.0, N_PER_ATOM)
Z_WELL = 4.0
PERTURB = 1e-3

_DIAMOND = np.array([
    [0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


def seed_for(index: int) -> int:
    return 9058000 + int(index)


def diamond_positions(tiling, rng: np.random.Generator, jitter: float = 0.1) -> np.ndarray:
    """Atom positions (bohr): 8-site diamond cell tiled n1 x n2 x n3, plus U(-j, j)^3 jitter."""
    n1, n2, n3 = tiling
    cells = np.array([[i, j, k] for i in range(n1) for j in range(n2) for k in range(n3)], float)
    pos = (cells[:, None, :] + _DIAMOND[None, :, :]).reshape(-1, 3) * A_BOHR
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    return pos


def _basis(pos: np.ndarray):
    """Centers and exponents of the 13 s-Gaussians on each atom (atom-major order)."""
    natoms = pos.shape[0]
    centers = np.repeat(pos, N_PER_ATOM, axis=0)
    alphas = np.tile(EXPONENTS, natoms)
    return centers, alphas


def _pair_blocks(ca, aa, cb, ab, shift, dev):
    """S and T for basis a (rows) against basis b translated by `shift` (columns)."""
    ca = torch.as_tensor(ca, dtype=torch.float64, device=dev)
    cb = torch.as_tensor(cb + shift[None, :], dtype=torch.float64, device=dev)
    aa = torch.as_tensor(aa, dtype=torch.float64, device=dev)
    ab = torch.as_tensor(ab, dtype=torch.float64, device=dev)
    d2 = torch.cdist(ca, cb).square_()
    p = aa[:, None] + ab[None, :]
    mu = aa[:, None] * ab[None, :] / p
    norm = (2.0 * aa / math.pi) ** 0.75
    normb = (2.0 * ab / math.pi) ** 0.75
    s = norm[:, None] * normb[None, :] * (math.pi / p) ** 1.5 * torch.exp(-mu * d2)
    t = mu * (3.0 - 2.0 * mu * d2) * s
    return s, t


def _well_overlaps(ca, aa, wells, shift, dev):
    """B_aC = <chi_a | exp(-|r - R_C - shift|^2)>."""
    ca = torch.as_tensor(ca, dtype=torch.float64, device=dev)
    wc = torch.as_tensor(wells + shift[None, :], dtype=torch.float64, device=dev)
    aa = torch.as_tensor(aa, dtype=torch.float64, device=dev)
    d2 = torch.cdist(ca, wc).square_()
    g = aa / (aa + 1.0)
    norm = (2.0 * aa / math.pi) ** 0.75
    return (norm * (math.pi / (aa + 1.0)) ** 1.5)[:, None] * torch.exp(-g[:, None] * d2)


def _sym_uniform(rng, n, dev):
    a = torch.as_tensor(rng.uniform(-1.0, 1.0, size=(n, n)), dtype=torch.float64, device=dev)
    return 0.5 * (a + a.T)


def _sus(S: torch.Tensor, U: torch.Tensor) -> torch.Tensor:
    """S U S for complex S and real symmetric U with real GEMMs (S U: two products;
    (S U) S: three products, (a+ib)(c+id) = ac - bd + i((a+b)(c+d) - ac - bd))."""
    a, b = S.real.contiguous(), S.imag.contiguous()
    pa, pb = a @ U, b @ U
    ac, bd = pa @ a, pb @ b
    mix = (pa + pb) @ (a + b)
    return torch.complex(ac - bd, mix - ac - bd)


def _hermitize(x: torch.Tensor) -> torch.Tensor:
    return 0.5 * (x + x.transpose(-1, -2).conj())


@dataclass
class Problem:
    """One generalized eigenproblem batch: H (nk, M, M), S (nk, N, N)."""
    H: torch.Tensor
    S: torch.Tensor
    n: int
    nk: int
    spin: str                 # "collinear" | "noncollinear" | "spin_polarized"
    kT: float
    n_elec: float
    kweights: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return 2 * self.n if self.spin == "noncollinear" else self.n

    @property
    def complex(self) -> bool:
        return self.H.is_complex()


def cluster(tiling, seed: int, device="cpu", jitter: float = 0.1):
    """Finite (Gamma-point, no images) cluster: real symmetric H, S of order 13 * atoms."""
    rng = np.random.default_rng(seed)
    pos = diamond_positions(tiling, rng, jitter)
    c, a = _basis(pos)
    zero = np.zeros(3)
    S, T = _pair_blocks(c, a, c, a, zero, device)
    B = _well_overlaps(c, a, pos, zero, device)
    V = -Z_WELL * (B @ B.T)
    U = _sym_uniform(rng, S.shape[0], device)
    H = T + V + PERTURB * (S @ U @ S)
    H = 0.5 * (H + H.T)
    S = 0.5 * (S + S.T)
    return H, S, pos, rng


def collinear_gamma(tiling, index: int, kT: float, n_elec: float | None = None, device="cpu") -> Problem:
    H, S, pos, _ = cluster(tiling, seed_for(index), device)
    natoms = pos.shape[0]
    ne = 4.0 * natoms if n_elec is None else n_elec
    return Problem(H[None], S[None], H.shape[0], 1, "collinear", kT, ne, np.ones(1),
                   name=f"cluster{tuple(tiling)}", meta={"atoms": natoms})


def mp_kpoints(mesh=(2, 2, 2)) -> np.ndarray:
    """Monkhorst-Pack fractions (units of the supercell reciprocal vectors)."""
    axes = [(2.0 * np.arange(1, m + 1) - m - 1) / (2.0 * m) for m in mesh]
    return np.array([[x, y, z] for x in axes[0] for y in axes[1] for z in axes[2]])


def lattice_images(L: np.ndarray, tol: float = 1e-18) -> list:
    """Supercell images n (integer 3-vectors) whose closest basis pair can still overlap:
    every image with min pair distance below sqrt(ln(1/tol)/mu_min) + 1 bohr is kept, so
    the Bloch sums drop no element above tol (a hard element cutoff makes S(k)
    indefinite).  For the 4x4x4 Si supercell this is the 27 nearest images."""
    amin = EXPONENTS.min()
    rcut = math.sqrt(math.log(1.0 / tol) / (0.5 * amin)) + 1.0
    nmax = [int(math.ceil(rcut / L[a])) + 1 for a in range(3)]
    out = []
    for i in range(-nmax[0], nmax[0] + 1):
        for j in range(-nmax[1], nmax[1] + 1):
            for k in range(-nmax[2], nmax[2] + 1):
                n = np.array([i, j, k])
                dmin = np.sqrt(np.sum(np.maximum(0.0, (np.abs(n) - 1) * L) ** 2))
                if dmin < rcut:
                    out.append(n)
    return out


def periodic(tiling, index: int, kT: float, n_elec: float | None = None, device="cpu",
             mesh=(2, 2, 2), kidx=None) -> Problem:
    """Bloch-summed H(k), S(k) (paper Sec. 2, Bloch-sum basis and S(k)) over the lattice
    images of `lattice_images` (27 for the 512-atom supercell), complex128 Hermitian per
    k-point; the S-sandwiched random term uses S(k) at each k.  kidx: build only these
    k-points of the mesh (the random draws do not depend on it; weights stay 1/nk_mesh)."""
    rng = np.random.default_rng(seed_for(index))
    pos = diamond_positions(tiling, rng)
    c, a = _basis(pos)
    n = c.shape[0]
    L = np.array(tiling, float) * A_BOHR
    kmesh = mp_kpoints(mesh)
    kf = kmesh if kidx is None else kmesh[list(kidx)]
    nk = kf.shape[0]
    images = lattice_images(L)
    Sk = torch.zeros(nk, n, n, dtype=torch.complex128, device=device)
    Hk = torch.zeros(nk, n, n, dtype=torch.complex128, device=device)
    Bk = torch.zeros(nk, n, pos.shape[0], dtype=torch.complex128, device=device)
    for img in images:
        shift = img * L
        phase = torch.as_tensor(np.exp(2j * np.pi * (kf @ img)), device=device)
        s, t = _pair_blocks(c, a, c, a, shift, device)
        # X(k)_lm = sum_T e^{i k.T} X_{l, m+T}
        Sk += phase[:, None, None] * s[None]
        Hk += phase[:, None, None] * t[None]
        del s, t
        b = _well_overlaps(c, a, pos, shift, device)
        Bk += phase[:, None, None] * b[None]
        del b
    U = _sym_uniform(rng, n, device)
    for ik in range(nk):
        Sk[ik] = _hermitize(Sk[ik])
        Hk[ik] += -Z_WELL * (Bk[ik] @ Bk[ik].conj().T)
        Hk[ik] += PERTURB * _sus(Sk[ik], U)
        Hk[ik] = _hermitize(Hk[ik])
    natoms = pos.shape[0]
    ne = 4.0 * natoms if n_elec is None else n_elec
    return Problem(Hk, Sk, n, nk, "collinear", kT, ne, np.full(nk, 1.0 / kmesh.shape[0]),
                   name=f"periodic{tuple(tiling)}k{nk}", meta={"atoms": natoms, "kpoints": kf})


def spinor_hamiltonian(H: torch.Tensor, S: torch.Tensor, moments: np.ndarray, KA: np.ndarray,
                       delta: float, lam: float, block: int = N_PER_ATOM) -> torch.Tensor:
    """Assemble the 2N x 2N spinor H_NC (paper Sec. 2 noncollinear GEP; Sec. 3.2 H_NC).

    H_NC = [[H + D Sz, D (Sx - i Sy) + l K], [D (Sx + i Sy) - l K, H - D Sz]] with the
    per-atom on-site terms taken in S-consistent form,
      S_q = S (blockdiag_A m_qA I_A) S = sum_A m_qA S[:, A] S[A, :],
      K   = S (blockdiag_A K_A) S,  K_A real antisymmetric, i.e. l i K (x) sigma_y.
    The basis functions are normalized (S_AA has a unit diagonal), so I_A stands for the
    diagonal of the atom's Gram block; its full inverse S_AA^-1 is left out on purpose:
    the same-centre Gaussian blocks have condition numbers near 1e12, and any evaluation of
    the inverse makes the pencil depend on the machine and library that build it at the
    1e-8 level, while these products of non-negative overlaps agree to a few rounding units.
    `block` is the number of basis functions per atom (13 for the Si basis)."""
    dev = H.device
    n = H.shape[0]
    m = torch.as_tensor(np.repeat(moments, block, axis=0), dtype=torch.float64, device=dev)  # (n, 3)
    Sq = [S @ (S * m[:, q:q + 1]) for q in range(3)]
    Sq = [0.5 * (x + x.T) for x in Sq]
    natoms = n // block
    Kb = torch.zeros(n, n, dtype=torch.float64, device=dev)
    for A in range(natoms):
        sl = slice(A * block, (A + 1) * block)
        Kb[sl, sl] = torch.as_tensor(KA[A], dtype=torch.float64, device=dev)
    Ks = S @ Kb @ S
    Ks = 0.5 * (Ks - Ks.T)
    Hc = H.to(torch.complex128)
    ab = delta * (Sq[0] - 1j * Sq[1]) + lam * Ks
    HN = torch.zeros(2 * n, 2 * n, dtype=torch.complex128, device=dev)
    HN[:n, :n] = Hc + delta * Sq[2]
    HN[n:, n:] = Hc - delta * Sq[2]
    HN[:n, n:] = ab
    HN[n:, :n] = ab.conj().T
    return _hermitize(HN)


def noncollinear(tiling, index: int, kT: float, n_elec: float | None = None, device="cpu",
                 delta: float = 0.05, lam: float = 0.01) -> Problem:
    """Gamma-point spinor problem on a cluster: seeded unit moments m_A (normalized
    Gaussian 3-vectors) and K_A = (B - B^T)/2, B ~ U(-1,1)^{13x13}.  S_NC = I_2 (x) S is
    implicit: only the N x N overlap is returned."""
    H, S, pos, rng = cluster(tiling, seed_for(index), device)
    natoms = pos.shape[0]
    m = rng.standard_normal((natoms, 3))
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    Kraw = rng.uniform(-1.0, 1.0, size=(natoms, N_PER_ATOM, N_PER_ATOM))
    KA = 0.5 * (Kraw - np.transpose(Kraw, (0, 2, 1)))
    HN = spinor_hamiltonian(H, S, m, KA, delta, lam)
    ne = 4.0 * natoms if n_elec is None else n_elec
    return Problem(HN[None], S.to(torch.complex128)[None], H.shape[0], 1, "noncollinear", kT, ne,
                   np.ones(1), name=f"nc{tuple(tiling)}",
                   meta={"atoms": natoms, "delta": delta, "lam": lam, "H": H, "S": S,
                         "moments": m, "KA": KA})


def spin_polarized(tiling, index: int, kT: float, n_elec: float | None = None, device="cpu",
                   delta: float = 0.05) -> Problem:
    """Collinear spin-polarized Gamma-point problem on a cluster: seeded per-atom moments
    m_A ~ U(-1, 1) along one axis and the S-consistent on-site exchange term of the
    noncollinear construction, H_up = H + D S_z, H_down = H - D S_z (S_z = S blockdiag(m_A
    I_A) S).  H is (1, 2, N, N) (channel after k), S (1, N, N)."""
    H, S, pos, rng = cluster(tiling, seed_for(index), device)
    natoms = pos.shape[0]
    m = np.zeros((natoms, 3))
    m[:, 2] = rng.uniform(-1.0, 1.0, natoms)
    HN = spinor_hamiltonian(H, S, m, np.zeros((natoms, N_PER_ATOM, N_PER_ATOM)), delta, 0.0).real
    n = H.shape[0]
    Hs = torch.stack([HN[:n, :n], HN[n:, n:]]).contiguous()
    ne = 4.0 * natoms if n_elec is None else n_elec
    return Problem(Hs[None], S[None], n, 1, "spin_polarized", kT, ne, np.ones(1), name=f"sp{tuple(tiling)}",
                   meta={"atoms": natoms, "delta": delta, "moments": m, "H": H, "S": S})


# ---------------------------------------------------------------------------------
# Closed-form test matrices (no randomness): used as pins for both sides.
# ---------------------------------------------------------------------------------

def chain(n: int, e0: float, t: float, s: float = 0.0):
    """1D chain: H tridiagonal (e0 on the diagonal, t off it), S = I + s * offdiag."""
    H = np.diag(np.full(n, e0)) + t * (np.eye(n, k=1) + np.eye(n, k=-1))
    S = np.eye(n) + s * (np.eye(n, k=1) + np.eye(n, k=-1))
    return H, S


def twisted_ring(n: int, e0: float, t: float, phi: float):
    """Periodic ring with a Peierls phase: H_{j,j+1} = t e^{i phi / n}."""
    H = np.zeros((n, n), complex)
    for j in range(n):
        H[j, j] = e0
        k = (j + 1) % n
        H[j, k] += t * np.exp(1j * phi / n)
        H[k, j] += t * np.exp(-1j * phi / n)
    return H, np.eye(n, dtype=complex)


def random_pencil(n: int, seed: int, complex_: bool = False, cond: float = 1e2):
    """Random Hermitian H and SPD S with a prescribed 2-norm condition number for S."""
    rng = np.random.default_rng(seed)
    if complex_:
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    else:
        A = rng.standard_normal((n, n))
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    H = 0.5 * (A + A.conj().T)
    sv = np.geomspace(1.0, 1.0 / cond, n)
    S = (Q * sv) @ Q.conj().T
    S = 0.5 * (S + S.conj().T)
    return H, S


def uneven_batch(seed: int = 4, count: int = 48, n_nc: int = 12, device="cpu") -> list:
    """Independent clusters with seeded tilings (n1, n2, n3) in {1..5}^3, 2 <= n1 n2 n3 <= 20
    (16-160 atoms, N = 208-2080); the first n_nc are noncollinear (2N up to 4160),
    the rest collinear real; kT 0.01, n_elec = 4 atoms."""
    rng = np.random.default_rng(seed_for(seed))
    tilings = []
    while len(tilings) < count:
        t = tuple(int(x) for x in rng.integers(1, 6, size=3))
        if 2 <= t[0] * t[1] * t[2] <= 20:
            tilings.append(t)
    out = []
    for b, t in enumerate(tilings):
        if b < n_nc:
            out.append(noncollinear(t, 100 + b, 0.01, device=device))
        else:
            out.append(collinear_gamma(t, 100 + b, 0.01, device=device))
    return out


def workload(name: str, device="cpu") -> Problem:
    """The named workloads (atom counts and N = 13 * atoms bind; see tiling notes)."""
    if name == "gamma64":       # 64 atoms, N = 832, real, kT 0.01, n_elec 256
        return collinear_gamma((2, 2, 2), 0, 0.01, 256.0, device)
    if name == "kbatch64":      # 64-atom supercell, N = 832, 8 k-points (small case of the same construction)
        return periodic((2, 2, 2), 1, 0.01, 256.0, device)
    if name == "kbatch512":     # 512 atoms, N = 6656, 8 k-points, complex, n_elec 2048
        return periodic((4, 4, 4), 1, 0.01, 2048.0, device)
    if name == "nc384":         # 384 atoms, N = 4992, 2N = 9984 spinor
        return noncollinear((4, 4, 3), 2, 0.01, 1536.0, device)
    if name == "adjoint216":    # 216 atoms, N = 2808, real, kT 0.02
        return collinear_gamma((3, 3, 3), 3, 0.02, 864.0, device)
    raise KeyError(name)
