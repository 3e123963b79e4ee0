"""Oracle results for the 48-system parity test (run as a script by fullsize_support).

Reads the pencils written to DIR, solves them with the plain CPU oracle (OpenMP over its
independent loops), and writes u.npz: per system the eigenvalues, the S-sandwiched density
matrix S rho S (what the test compares, S-covariantly), mu, E_band and the condition
numbers beta_i of the eigenvalues."""
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


if __name__ == "__main__":
    main(sys.argv[1])
