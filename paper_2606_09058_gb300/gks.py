"""Python binding of the C ABI in include/gks.h (argument marshalling only).

Every step of the path runs in libgks.so; PyTorch supplies device memory and the CUDA
stream.  The binding refuses to run without the compiled library or a CUDA device.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

GKS_OK, GKS_EINVAL, GKS_ENOTSPD, GKS_ENOCONV, GKS_ENOMEM, GKS_ECUDA, GKS_ETIMEOUT, GKS_ENOTIMPL = range(8)
GKS_R64, GKS_C128 = 0, 1
GKS_COLLINEAR, GKS_NONCOLLINEAR, GKS_SPIN_POLARIZED = 0, 1, 2
GKS_FP64, GKS_MIXED_TF32, GKS_MIXED_SPLITBF16 = 0, 1, 2
GKS_REUSE_S_FACTOR, GKS_SAVE_FOR_BACKWARD, GKS_EIGEN_ONLY = 1, 2, 4
GKS_DEBUG_SKIP_COPY = 1
GKS_SPLIT_RESIDUES, GKS_SPLIT_DIGITS = 0, 1
GKS_HEMV_DIGITS, GKS_HEMV_FP64 = 0, 1
_SPIN = {"collinear": GKS_COLLINEAR, "noncollinear": GKS_NONCOLLINEAR, "spin_polarized": GKS_SPIN_POLARIZED}
_PREC = {"fp64": GKS_FP64, "mixed_tf32": GKS_MIXED_TF32, "mixed": GKS_MIXED_SPLITBF16,
         "mixed_splitbf16": GKS_MIXED_SPLITBF16}
_NAMES = {0: "GKS_OK", 1: "GKS_EINVAL", 2: "GKS_ENOTSPD", 3: "GKS_ENOCONV", 4: "GKS_ENOMEM", 5: "GKS_ECUDA",
          6: "GKS_ETIMEOUT", 7: "GKS_ENOTIMPL"}

_lib = None


class GKSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("precision", ctypes.c_int),
                ("f_cut", ctypes.c_double), ("profile", ctypes.c_int), ("graph", ctypes.c_int),
                ("gemm", ctypes.c_int), ("slices", ctypes.c_int), ("block", ctypes.c_int),
                ("refine_sweeps", ctypes.c_int), ("n_ev", ctypes.c_int), ("wait_limit", ctypes.c_longlong),
                ("autotune_cache", ctypes.c_char_p), ("debug", ctypes.c_int), ("reduction", ctypes.c_int),
                ("tridiag", ctypes.c_int), ("band", ctypes.c_int), ("split", ctypes.c_int),
                ("hemv", ctypes.c_int)]


class _Problem(ctypes.Structure):
    _fields_ = [("H", ctypes.c_void_p), ("S", ctypes.c_void_p), ("n", ctypes.c_int64), ("nk", ctypes.c_int64),
                ("dtype", ctypes.c_int), ("spin_mode", ctypes.c_int), ("kT", ctypes.c_double),
                ("n_elec", ctypes.c_double), ("kweights", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("rho", ctypes.c_void_p),
                ("e_band", ctypes.c_void_p)]


class _ProfEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("groups", ctypes.c_int), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libgks.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I64, D, I, U = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_uint
    lib.gks_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_Opts)]
    lib.gks_destroy.argtypes = [P]
    lib.gks_last_error.argtypes = [P]
    lib.gks_last_error.restype = ctypes.c_char_p
    lib.gks_solve.argtypes = [P, P, P, I64, I64, I, I, D, D, P, U, P, P, P, P, P]
    lib.gks_sync.argtypes = [P]
    lib.gks_potrf.argtypes = [P, P, I64, I64, I]
    lib.gks_reduce.argtypes = [P, P, P, I64, I64, I]
    lib.gks_stedc.argtypes = [P, P, P, I64, I64, P, P]
    lib.gks_gemm.argtypes = [P, I, I, I, I64, I64, I64, D, P, I64, P, I64, D, P, I64, I]
    lib.gks_gemm.restype = I
    lib.gks_gemm_split_noalloc.argtypes = [P, I, I, I, I64, I64, I64, D, P, I64, P, I64, D, P, I64]
    lib.gks_gemm_split_noalloc.restype = I
    lib.gks_tune.argtypes = [P, I64, I64, I, I, ctypes.POINTER(ctypes.c_int), I, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int)]
    lib.gks_tune.restype = I
    lib.gks_tune_set.argtypes = [P, I64, I, I, I]
    lib.gks_tune_set.restype = I
    lib.gks_tune_get.argtypes = [P, I64, I, I]
    lib.gks_tune_get.restype = I
    lib.gks_solve_batched.argtypes = [P, I64, ctypes.POINTER(_Problem), I]
    lib.gks_solve_batched.restype = I
    lib.gks_adjoint.argtypes = [P, P, P, P, I64, I64, I, I, D, P, P, P, D, P, P]
    lib.gks_adjoint.restype = I
    lib.gks_occupy.argtypes = [P, P, I64, I64, P, I64, I64, I, I, D, D, P, P, P, P, P]
    lib.gks_occupy.restype = I
    lib.gks_profile.argtypes = [P, ctypes.POINTER(_ProfEntry), I]
    lib.gks_profile.restype = I
    lib.gks_he2hb.argtypes = [P, P, I64, I64, I, I, P]
    lib.gks_he2hb.restype = I
    lib.gks_hb2st.argtypes = [P, P, I64, I64, I, I, P, P, P, I64]
    lib.gks_hb2st.restype = I
    lib.gks_refine_stats.argtypes = [P, ctypes.POINTER(ctypes.c_double), I]
    lib.gks_refine_stats.restype = I
    lib.gks_measure_peak.argtypes = [P, I, ctypes.POINTER(ctypes.c_double)]
    lib.gks_measure_peak.restype = I
    lib.gks_launch_count.argtypes = []
    lib.gks_launch_count.restype = ctypes.c_longlong
    for f in ("gks_create", "gks_destroy", "gks_solve", "gks_sync", "gks_potrf", "gks_reduce", "gks_stedc"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_tensor(t: torch.Tensor, name: str, dtypes):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclass
class Solution:
    eps: torch.Tensor      # (nk, M) float64, ascending
    C: torch.Tensor        # (nk, M, M)
    mu: torch.Tensor       # (1,) float64
    rho: torch.Tensor      # (nk, M, M)
    e_band: torch.Tensor   # (1,) float64


class Context:
    """A gks context bound to one device and one CUDA stream."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None, f_cut: float = 1e-16,
                 profile: bool = False, graph: bool = False, gemm: str = "auto", slices: int = 0,
                 block: int = 0, precision: str = "fp64", refine_sweeps: int = 0, n_ev: int = 0,
                 wait_limit: int = 0, autotune_cache: str | None = None, debug: int = 0,
                 reduction: str = "cholesky", tridiag: str = "one_stage", band: int = 0,
                 split: str = "residues", hemv: str = "digits"):
        if not torch.cuda.is_available():
            raise RuntimeError("gks needs a CUDA device")
        lib = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        gm = {"auto": 0, "fp64": 1, "split": 2}[gemm]
        self.n_ev = int(n_ev)
        self.precision = precision
        cache = autotune_cache.encode() if autotune_cache else None
        opts = _Opts(self.device, ctypes.c_void_p(self.stream.cuda_stream), _PREC[precision], f_cut,
                     1 if profile else 0, 1 if graph else 0, gm, int(slices), int(block), int(refine_sweeps),
                     int(n_ev), int(wait_limit), cache, int(debug), {"cholesky": 0, "lowdin": 1}[reduction],
                     {"one_stage": 0, "two_stage": 1}[tridiag], int(band),
                     {"residues": GKS_SPLIT_RESIDUES, "digits": GKS_SPLIT_DIGITS}[split],
                     {"digits": GKS_HEMV_DIGITS, "fp64": GKS_HEMV_FP64}[hemv])
        h = ctypes.c_void_p()
        rc = lib.gks_create(ctypes.byref(h), ctypes.byref(opts))
        if rc:
            raise GKSError(rc, "gks_create failed")
        self._h = h
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, rc):
        if rc:
            raise GKSError(rc, self._lib.gks_last_error(self._h).decode())

    def sync(self):
        self._raise(self._lib.gks_sync(self._h))

    def profile(self) -> list[dict]:
        """Event profile since the previous call: kernel classes and stages with device
        time (ms) and algorithmic flops/bytes (empty unless created with profile=True)."""
        buf = (_ProfEntry * 64)()
        n = self._lib.gks_profile(self._h, buf, 64)
        return [dict(name=buf[i].name.decode(), groups=buf[i].groups, ms=buf[i].ms, flops=buf[i].flops,
                     bytes=buf[i].bytes) for i in range(n)]

    # ------------------------------------------------------------------ full path
    def _ncols(self, M: int) -> int:
        return self.n_ev if 0 < self.n_ev < M else M

    @staticmethod
    def _flags(reuse_s: bool, save: bool, eigen_only: bool) -> int:
        return ((GKS_REUSE_S_FACTOR if reuse_s else 0) | (GKS_SAVE_FOR_BACKWARD if save else 0)
                | (GKS_EIGEN_ONLY if eigen_only else 0))

    def solve_into(self, H, S, kT, n_elec, spin="collinear", kweights=None, *, eps, C, mu=None, rho=None,
                   e_band=None, sync=True, reuse_s=False, save_for_backward=False, eigen_only=False):
        """gks_solve on caller-provided output tensors (no allocation)."""
        nk = H.shape[0]
        n = S.shape[-1]
        dt = GKS_C128 if H.is_complex() else GKS_R64
        rc = self._lib.gks_solve(self._h, _ptr(H), _ptr(S), n, nk, dt, _SPIN[spin], float(kT), float(n_elec),
                                 _ptr(kweights), self._flags(reuse_s, save_for_backward, eigen_only), _ptr(eps),
                                 _ptr(C), _ptr(mu), _ptr(rho), _ptr(e_band))
        self._raise(rc)
        if sync:
            self.sync()

    def solve(self, H: torch.Tensor, S: torch.Tensor, kT: float, n_elec: float, spin: str = "collinear",
              kweights: torch.Tensor | None = None, sync: bool = True, reuse_s: bool = False,
              save_for_backward: bool = False, eigen_only: bool = False) -> Solution:
        """eps, C, mu, rho, E_band for nk pencils sharing one chemical potential.

        H: (nk, M, M), S: (nk, n, n) (noncollinear: M = 2n, S the n x n overlap;
        spin_polarized: H (nk, 2, n, n), eps (nk, 2, n), C and rho (nk, 2, n, n)).  With
        n_ev set on the context C keeps only its leading n_ev columns."""
        sp = spin == "spin_polarized"
        if H.dim() == (3 if sp else 2):
            H, S = H[None], S[None]
        cd = (torch.float64, torch.complex128)
        _check_tensor(H, "H", cd)
        _check_tensor(S, "S", cd)
        if S.dtype != H.dtype:
            raise ValueError("H and S must share a dtype")
        nk, M = H.shape[0], H.shape[-1]
        lead = (nk, 2) if sp else (nk,)
        if kweights is not None:
            _check_tensor(kweights, "kweights", (torch.float64,))
        dev = H.device
        eps = torch.empty(*lead, M, dtype=torch.float64, device=dev)
        C = torch.empty(*lead, M, self._ncols(M), dtype=H.dtype, device=dev)
        rho = None if eigen_only else torch.empty(*lead, M, M, dtype=H.dtype, device=dev)
        mu = None if eigen_only else torch.empty(1, dtype=torch.float64, device=dev)
        eb = None if eigen_only else torch.empty(1, dtype=torch.float64, device=dev)
        self.solve_into(H, S, kT, n_elec, spin, kweights, eps=eps, C=C, mu=mu, rho=rho, e_band=eb, sync=sync,
                        reuse_s=reuse_s, save_for_backward=save_for_backward, eigen_only=eigen_only)
        return Solution(eps, C, mu, rho, eb)

    def occupy(self, eps_all: torch.Tensor, C: torch.Tensor | None, kT: float, n_elec: float, k0: int = 0,
               spin: str = "collinear", kweights_all: torch.Tensor | None = None, rho: bool = True,
               edm: bool = False, sync: bool = True):
        """gks_occupy: mu shared by every k-point of eps_all (nk_all, M) (spin_polarized:
        (nk_all, 2, n)), then the density matrix and optionally the energy-density matrix
        of the local k-points k0 .. k0 + nk - 1 whose eigenvectors are C.  Returns
        (mu, rho, e_band, edm)."""
        _check_tensor(eps_all, "eps_all", (torch.float64,))
        sp = spin == "spin_polarized"
        nk_all = eps_all.shape[0]
        M = eps_all.shape[-1]
        n = M // 2 if spin == "noncollinear" else M
        dev = eps_all.device
        nk = 0 if C is None else C.shape[0]
        lead = (nk, 2) if sp else (nk,)
        dt = torch.complex128 if (C is not None and C.is_complex()) else torch.float64
        mu = torch.empty(1, dtype=torch.float64, device=dev)
        eb = torch.empty(1, dtype=torch.float64, device=dev)
        r = torch.empty(*lead, M, M, dtype=dt, device=dev) if (rho and nk) else None
        e = torch.empty(*lead, M, M, dtype=dt, device=dev) if (edm and nk) else None
        rc = self._lib.gks_occupy(self._h, _ptr(eps_all), nk_all, int(k0), _ptr(C), n, nk,
                                  GKS_C128 if dt == torch.complex128 else GKS_R64, _SPIN[spin], float(kT),
                                  float(n_elec), _ptr(kweights_all), _ptr(mu), _ptr(r), _ptr(eb), _ptr(e))
        self._raise(rc)
        if sync:
            self.sync()
        return mu, r, eb, e

    # ------------------------------------------------------------------ batch
    def solve_batched(self, problems, nstreams: int = 8, sync: bool = True, out: list | None = None) -> list:
        """Independent problems of uneven order in one launch sequence.  `problems` is a list
        of dicts with keys H, S, kT, n_elec and optional spin, kweights; returns one
        Solution per problem (allocated here unless `out` passes those of a previous call;
        reusing them lets a graph-mode context replay its captured batch)."""
        arr = (_Problem * len(problems))()
        sols = []
        for b, pr in enumerate(problems):
            H, S = pr["H"], pr["S"]
            if H.dim() == 2:
                H, S = H[None], S[None]
            spin = pr.get("spin", "collinear")
            nk, M = H.shape[0], H.shape[1]
            dev = H.device
            sol = out[b] if out is not None else Solution(
                torch.empty(nk, M, dtype=torch.float64, device=dev),
                torch.empty(nk, M, self._ncols(M), dtype=H.dtype, device=dev),
                torch.empty(1, dtype=torch.float64, device=dev), torch.empty(nk, M, M, dtype=H.dtype, device=dev),
                torch.empty(1, dtype=torch.float64, device=dev))
            kw = pr.get("kweights")
            arr[b] = _Problem(H.data_ptr(), S.data_ptr(), S.shape[-1], nk, GKS_C128 if H.is_complex() else GKS_R64,
                              _SPIN[spin], float(pr["kT"]),
                              float(pr["n_elec"]), kw.data_ptr() if kw is not None else None, sol.eps.data_ptr(),
                              sol.C.data_ptr(), sol.mu.data_ptr(), sol.rho.data_ptr(), sol.e_band.data_ptr())
            sols.append(sol)
        self._keep = (problems, sols)
        self._raise(self._lib.gks_solve_batched(self._h, len(problems), arr, nstreams))
        if sync:
            self.sync()
        return sols

    # ------------------------------------------------------------------ adjoint
    def adjoint(self, sol: Solution | None, S: torch.Tensor, kT: float, spin: str = "collinear", kweights=None,
                rho_bar: torch.Tensor | None = None, eps_bar: torch.Tensor | None = None,
                e_band_bar: float = 0.0, sync: bool = True, complex_: bool | None = None):
        """Gradients (H_bar, S_bar) of L(rho, eps, E_band) through a previous solve (n_elec
        fixed): dL = Re tr(H_bar^H dH) + Re tr(S_bar^H dS) for Hermitian dH, dS.  sol = None
        uses the eigenpairs the context kept from its last solve with save_for_backward."""
        n = S.shape[-1]
        nk = S.shape[0] if S.dim() == 3 else 1
        sp = spin == "spin_polarized"
        M = 2 * n if spin == "noncollinear" else n
        if sol is not None:
            C, eps, mu = sol.C, sol.eps, sol.mu
            dt = C.dtype
        else:
            C = eps = mu = None
            dt = S.dtype if complex_ is None else (torch.complex128 if complex_ else torch.float64)
        for t, nm in ((rho_bar, "rho_bar"), (eps_bar, "eps_bar")):
            if t is not None:
                _check_tensor(t, nm, (torch.float64, torch.complex128))
        lead = (nk, 2) if sp else (nk,)
        Hb = torch.empty(*lead, M, M, dtype=dt, device=S.device)
        Sb = torch.empty(nk, n, n, dtype=dt, device=S.device)
        rc = self._lib.gks_adjoint(self._h, _ptr(C), _ptr(eps), _ptr(mu), n, nk,
                                   GKS_C128 if dt == torch.complex128 else GKS_R64, _SPIN[spin], float(kT),
                                   _ptr(kweights), _ptr(rho_bar), _ptr(eps_bar), float(e_band_bar), _ptr(Hb),
                                   _ptr(Sb))
        self._raise(rc)
        if sync:
            self.sync()
        return Hb, Sb

    def refine_stats(self):
        """Per sweep and item of the last mixed-precision solve: (bound on ||I - X^H X||,
        bound on ||X^H H' X - diag(l)||) at the start of the sweep, as an array
        (sweeps * items, 2) in sweep-major order."""
        import numpy as np
        buf = (ctypes.c_double * 4096)()
        n = self._lib.gks_refine_stats(self._h, buf, 4096)
        a = np.array(buf[:n])
        return a.reshape(-1, 2)

    def measure_peak(self, unit: str = "dfma") -> float:
        """gks_measure_peak: measured TFLOP/s of the FP64 FMA pipe ("dfma") or of the FP64
        mma.sync instruction ("dmma") on this device."""
        out = ctypes.c_double()
        self._raise(self._lib.gks_measure_peak(self._h, {"dfma": 0, "dmma": 1}[unit], ctypes.byref(out)))
        return out.value

    # ------------------------------------------------------------------ stages
    def gemm(self, A, B, C, opA="N", opB="N", alpha=1.0, beta=0.0, mode="split"):
        """C = alpha op(A) op(B) + beta C through gks_gemm (mode "fp64" or "split")."""
        ops = {"N": 0, "T": 1, "C": 2}
        M, N = C.shape
        K = A.shape[1] if opA == "N" else A.shape[0]
        rc = self._lib.gks_gemm(self._h, GKS_C128 if C.is_complex() else GKS_R64, ops[opA], ops[opB], M, N, K,
                                float(alpha), _ptr(A), A.shape[1], _ptr(B), B.shape[1], float(beta), _ptr(C),
                                C.shape[1], 1 if mode == "fp64" else 2)
        self._raise(rc)
        self.sync()
        return C

    def tune(self, n: int, nk: int = 1, complex_: bool = False, spin: str = "collinear",
             widths=(128, 256, 384, 512)) -> tuple[int, dict]:
        """gks_tune: time the candidate outer widths on seeded pencils of this shape and keep
        the fastest for the shape class; returns (best width, {width: ms})."""
        w = (ctypes.c_int * len(widths))(*widths)
        ms = (ctypes.c_double * len(widths))()
        best = ctypes.c_int()
        rc = self._lib.gks_tune(self._h, int(n), int(nk), GKS_C128 if complex_ else GKS_R64,
                                1 if spin == "noncollinear" else 0, w, len(widths), ms, ctypes.byref(best))
        self._raise(rc)
        return best.value, {int(widths[i]): ms[i] for i in range(len(widths))}

    def tune_set(self, n: int, complex_: bool, spin: str, width: int):
        self._raise(self._lib.gks_tune_set(self._h, int(n), GKS_C128 if complex_ else GKS_R64,
                                           1 if spin == "noncollinear" else 0, int(width)))

    def tune_get(self, n: int, complex_: bool = False, spin: str = "collinear") -> int:
        return self._lib.gks_tune_get(self._h, int(n), GKS_C128 if complex_ else GKS_R64,
                                      1 if spin == "noncollinear" else 0)

    def gemm_split_noalloc(self, A, B, C, opA="N", opB="N", alpha=1.0, beta=0.0):
        """C = alpha op(A) op(B) + beta C through gks_gemm_split_noalloc: the split product
        on the library's fixed device scratch, with no device allocation."""
        ops = {"N": 0, "T": 1, "C": 2}
        M, N = C.shape
        K = A.shape[1] if opA == "N" else A.shape[0]
        rc = self._lib.gks_gemm_split_noalloc(self._h, GKS_C128 if C.is_complex() else GKS_R64, ops[opA], ops[opB],
                                              M, N, K, float(alpha), _ptr(A), A.shape[1], _ptr(B), B.shape[1],
                                              float(beta), _ptr(C), C.shape[1])
        self._raise(rc)
        self.sync()
        return C

    def potrf(self, A: torch.Tensor) -> torch.Tensor:
        """In place lower Cholesky factor of each (count, m, m) matrix."""
        if A.dim() == 2:
            A = A[None]
        _check_tensor(A, "A", (torch.float64, torch.complex128))
        rc = self._lib.gks_potrf(self._h, _ptr(A), A.shape[1], A.shape[0], GKS_C128 if A.is_complex() else GKS_R64)
        self._raise(rc)
        self.sync()
        return A

    def reduce(self, H: torch.Tensor, S: torch.Tensor):
        """In place: S <- L, lower(H) <- lower(L^-1 H L^-H)."""
        if H.dim() == 2:
            H, S = H[None], S[None]
        for t, nm in ((H, "H"), (S, "S")):
            _check_tensor(t, nm, (torch.float64, torch.complex128))
        rc = self._lib.gks_reduce(self._h, _ptr(H), _ptr(S), H.shape[1], H.shape[0],
                                  GKS_C128 if H.is_complex() else GKS_R64)
        self._raise(rc)
        self.sync()
        return H, S

    def he2hb(self, A: torch.Tensor, band: int, want_q: bool = False):
        """Stage 1 of the two-stage reduction in place on A (count, m, m): A <- band matrix
        B = Q1^H A Q1 (full Hermitian storage); returns (B, Q1 or None)."""
        if A.dim() == 2:
            A = A[None]
        _check_tensor(A, "A", (torch.float64, torch.complex128))
        Q = torch.empty_like(A) if want_q else None
        self._raise(self._lib.gks_he2hb(self._h, _ptr(A), A.shape[1], A.shape[0],
                                        GKS_C128 if A.is_complex() else GKS_R64, int(band), _ptr(Q)))
        self.sync()
        return A, Q

    def hb2st(self, B: torch.Tensor, band: int, X: torch.Tensor | None = None):
        """Stage 2: (d, e) of the real tridiagonal Q2^H B Q2 for the Hermitian band B
        (count, m, m); X (count, m, ncols) is replaced by Q2 X when given."""
        if B.dim() == 2:
            B = B[None]
        _check_tensor(B, "B", (torch.float64, torch.complex128))
        count, m = B.shape[0], B.shape[1]
        d = torch.empty(count, m, dtype=torch.float64, device=B.device)
        e = torch.empty(count, m, dtype=torch.float64, device=B.device)
        nc = 0 if X is None else X.shape[-1]
        self._raise(self._lib.gks_hb2st(self._h, _ptr(B), m, count, GKS_C128 if B.is_complex() else GKS_R64,
                                        int(band), _ptr(d), _ptr(e), _ptr(X), nc))
        self.sync()
        return d, e

    def stedc(self, d: torch.Tensor, e: torch.Tensor):
        """Divide-and-conquer eigensolve of real tridiagonals d (count, m), e (count, m)."""
        if d.dim() == 1:
            d, e = d[None], e[None]
        _check_tensor(d, "d", (torch.float64,))
        _check_tensor(e, "e", (torch.float64,))
        count, m = d.shape
        lam = torch.empty(count, m, dtype=torch.float64, device=d.device)
        Z = torch.empty(count, m, m, dtype=torch.float64, device=d.device)
        rc = self._lib.gks_stedc(self._h, _ptr(d), _ptr(e), m, count, _ptr(lam), _ptr(Z))
        self._raise(rc)
        self.sync()
        return lam, Z


def launch_count() -> int:
    """Kernel launches issued by libgks.so in this process."""
    return int(load().gks_launch_count())


_default: dict = {}


def context(device: int | None = None) -> Context:
    """A cached context for the current device and stream."""
    dev = torch.cuda.current_device() if device is None else device
    key = (dev, torch.cuda.current_stream(dev).cuda_stream)
    if key not in _default:
        _default[key] = Context(dev)
    return _default[key]


def solve(H, S, kT, n_elec, spin="collinear", kweights=None) -> Solution:
    return context(H.device.index).solve(H, S, kT, n_elec, spin, kweights)


class GKSSolve(torch.autograd.Function):
    """eps, rho, E_band, mu = GKSSolve.apply(H, S, kT, n_elec, spin, kweights, recompute).

    Forward runs gks_solve; backward runs gks_adjoint (n_elec fixed).  H and S must be
    Hermitian (the solver reads their lower triangles); the gradients returned are the
    Hermitian ones, i.e. those of a loss evaluated on Hermitian H and S.

    recompute=True keeps no eigenvectors between forward and backward: backward solves the
    saved H, S again and then runs the adjoint.  Cost: one more full solve in backward.
    Memory: the nk M^2 elements of C are not held, but H (the same element count) is; the
    saving is real only when the caller keeps H alive anyway (it usually does, as the
    graph input).  The solve is deterministic for a fixed outer width, so the second solve
    reproduces the forward's C, eps and mu bit for bit; the width in effect at forward is
    recorded, and backward raises if it has changed in between (a gks_tune or tune_set of
    that shape class)."""

    @staticmethod
    def forward(ctx, H, S, kT, n_elec, spin="collinear", kweights=None, recompute=False):
        c = context(H.device.index)
        Hb = (H if H.dim() == 3 else H[None]).contiguous()
        Sb = (S if S.dim() == 3 else S[None]).contiguous()
        sol = c.solve(Hb, Sb, kT, n_elec, spin, kweights)
        if recompute:
            ctx.save_for_backward(Hb, Sb)
            ctx.width = c.tune_get(Sb.shape[-1], Hb.is_complex(), spin)
        else:
            ctx.save_for_backward(sol.C, sol.eps, sol.mu, Sb)
        ctx.recompute = bool(recompute)
        ctx.kT, ctx.n_elec, ctx.spin, ctx.kweights = kT, n_elec, spin, kweights
        ctx.hshape, ctx.sshape = H.shape, S.shape
        ctx.mark_non_differentiable(sol.mu)
        return sol.eps, sol.rho, sol.e_band, sol.mu

    @staticmethod
    def backward(ctx, g_eps, g_rho, g_eband, g_mu):
        if ctx.recompute:
            Hb, Sb = ctx.saved_tensors
            c = context(Hb.device.index)
            if c.tune_get(Sb.shape[-1], Hb.is_complex(), ctx.spin) != ctx.width:
                raise RuntimeError("GKSSolve(recompute=True): the outer block width of this shape class changed "
                                   "between forward and backward, so the recomputed eigenvectors would differ")
            sol = c.solve(Hb, Sb, ctx.kT, ctx.n_elec, ctx.spin, ctx.kweights)
        else:
            C, eps, mu, Sb = ctx.saved_tensors
            c = context(C.device.index)
            sol = Solution(eps, C, mu, None, None)
        eb = 0.0 if g_eband is None else float(g_eband.reshape(-1)[0].item())
        Hbar, Sbar = c.adjoint(sol, Sb, ctx.kT, ctx.spin, ctx.kweights,
                               rho_bar=None if g_rho is None else g_rho.contiguous(),
                               eps_bar=None if g_eps is None else g_eps.contiguous(), e_band_bar=eb)
        return Hbar.reshape(ctx.hshape), Sbar.reshape(ctx.sshape), None, None, None, None, None
