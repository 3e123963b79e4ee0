"""Oracle results for the full-size parity tests (run as a script by fullsize_support).

Reads the pencils written to DIR, solves them with the plain CPU oracle (OpenMP over its
independent loops), and writes one .npz per case: eigenvalues, the S-sandwiched density
matrix S rho S (what the tests compare, S-covariantly), mu, E_band and the condition
numbers beta_i of the eigenvalues.  Cases in order: the 48 uneven systems (u.npz), then
k-point 0 of the 512-atom k-batch solved as a pencil of its own (kbatch512_k0.npz)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402


def _save(d, name, **arrays):
    tmp = os.path.join(d, name + ".tmp.npz")
    np.savez(tmp, **arrays)
    os.replace(tmp, os.path.join(d, name + ".npz"))


def main(d):
    meta = np.load(os.path.join(d, "meta.npy"), allow_pickle=True).item()
    O.build()
    t0 = time.time()
    out = {}
    for b, (kT, ne, spin) in enumerate(meta["u"]):
        H = np.load(os.path.join(d, f"u{b}_H.npy"))
        S = np.load(os.path.join(d, f"u{b}_S.npy"))
        r = O.solve(H[None], S[None], kT, ne, spin)
        Sk = O.spinor_overlap(S) if spin == "noncollinear" else S
        beta = O.eig_condition(H, Sk, r.eps[0], r.C[0], (O.hermitian_norm2(H), O.hermitian_norm2(Sk)))
        out[f"eps{b}"] = r.eps[0]
        out[f"srs{b}"] = Sk @ r.rho[0] @ Sk
        out[f"beta{b}"] = beta
        out[f"mu{b}"] = np.array(r.mu)
        out[f"eb{b}"] = np.array(r.e_band)
        print(f"system {b}: M={H.shape[0]} {time.time() - t0:.1f} s", flush=True)
    _save(d, "u", **out)
    # k-point 0 of the 512-atom k-batch as a pencil of its own (its own mu for the same
    # electron count per k-point: the shared mu needs all eight k-points)
    kT, ne, spin = meta["kb"]
    H = np.load(os.path.join(d, "kb_H0.npy"))
    S = np.load(os.path.join(d, "kb_S0.npy"))
    t1 = time.time()
    r = O.solve(H[None], S[None], kT, ne, spin)
    t2 = time.time()
    beta = O.eig_condition(H, S, r.eps[0], r.C[0], (O.hermitian_norm2(H), O.hermitian_norm2(S)))
    _save(d, "kbatch512_k0", eps=r.eps[0], srs=S @ r.rho[0] @ S, beta=beta, mu=np.array(r.mu),
          eb=np.array(r.e_band), seconds=np.array(t2 - t1),
          threads=np.array(int(os.environ.get("OMP_NUM_THREADS", "1"))))
    print(f"kbatch512 k0: M={H.shape[0]} solve {t2 - t1:.1f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1])
