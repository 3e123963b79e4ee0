"""Write the oracle results the full-size parity tests and the benchmark's accuracy check
compare against (run on the host cores; it takes about an hour on eight cores):

* kbatch512_oracle.npz: the 512-atom supercell (N = 6656), k-points 0..3 of the 2x2x2
  Monkhorst-Pack mesh (one of each time-reversal pair k, -k; the other four have the same
  spectrum): eigenvalues and their condition numbers beta_i; k-point 0 also solved as a
  pencil of its own with n_elec = 2048 (mu, E_band, and S rho S on sampled entries).
* nc384_oracle.npz: the 384-atom noncollinear cluster (2N = 9984): eigenvalues, beta_i,
  mu, E_band, S_NC rho S_NC on sampled entries.

Inputs come from paper_2606_09058_gb300.inputs built on the CPU; every stored value comes
from oracle/ (this script calls nothing else).  The CUDA tests build the same pencils on
the GPU, which agree with these to a few units of FP64 rounding; the eigenvalue gates
max(1e-10, 8 beta_i) are first-order bounds for perturbations of that size.

Sampled entries: the diagonal and 4096 (row, column) pairs drawn with numpy PCG64 seed
9058100 (kbatch512) or 9058101 (nc384)."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2606_09058_gb300 import inputs as I  # noqa: E402


def samples(M, seed, count=4096):
    rng = np.random.default_rng(seed)
    i = np.concatenate([np.arange(M), rng.integers(0, M, count)]).astype(np.int32)
    j = np.concatenate([np.arange(M), rng.integers(0, M, count)]).astype(np.int32)
    return i, j


def sampled_srs(S, rho, i, j):
    """(S rho S)[i, j] for the sampled pairs without forming the full product."""
    A = S[i, :] @ rho               # rows i of S rho
    return np.einsum("pk,kp->p", A, S[:, j])


def kbatch512(out):
    res = {}
    for k in range(4):
        t = time.time()
        p = I.periodic((4, 4, 4), 1, 0.01, 2048.0, kidx=[k])
        H, S = p.H[0].numpy(), p.S[0].numpy()
        if k == 0:
            r = O.solve(H[None], S[None], p.kT, p.n_elec)
            eps, C = r.eps[0], r.C[0]
            i, j = samples(H.shape[0], 9058100)
            res.update(k0_mu=np.array(r.mu), k0_eb=np.array(r.e_band), k0_i=i, k0_j=j,
                       k0_srs=sampled_srs(S, r.rho[0], i, j))
        else:
            eps, C = O.eigh_generalized(H, S)
        res[f"eps{k}"] = eps
        res[f"beta{k}"] = O.eig_condition(H, S, eps, C, (O.hermitian_norm2(H), O.hermitian_norm2(S)))
        print(f"kbatch512 k={k}: {time.time() - t:.0f} s", flush=True)
        np.savez_compressed(out, **res)


def nc384(out):
    t = time.time()
    p = I.workload("nc384")
    H, S = p.H[0].numpy(), p.S[0].numpy()
    r = O.solve(H[None], S[None], p.kT, p.n_elec, "noncollinear")
    Sn = O.spinor_overlap(S)
    i, j = samples(H.shape[0], 9058101)
    np.savez_compressed(out, eps=r.eps[0], mu=np.array(r.mu), eb=np.array(r.e_band), i=i, j=j,
                        srs=sampled_srs(Sn, r.rho[0], i, j),
                        beta=O.eig_condition(H, Sn, r.eps[0], r.C[0], (O.hermitian_norm2(H), O.hermitian_norm2(Sn))))
    print(f"nc384: {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["kbatch512", "nc384"]
    if "kbatch512" in which:
        kbatch512(os.path.join(HERE, "kbatch512_oracle.npz"))
    if "nc384" in which:
        nc384(os.path.join(HERE, "nc384_oracle.npz"))
