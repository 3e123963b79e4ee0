#!/usr/bin/env python
"""Benchmark of the generalized Kohn-Sham eigensolve + density matrix on one GB300.

Workload (default "kbatch512"): the 512-atom Si supercell (4x4x4 conventional cells,
N = 13 * 512 = 6656 s-Gaussians), complex128 Bloch-summed H(k), S(k) at the 8
Monkhorst-Pack k-points, kT = 0.01 Ha, n_elec = 2048, one chemical potential shared by
all k-points, FP64 throughout.  One step = one gks_solve of the whole k-batch
(Cholesky, reduction, tridiagonalization, divide and conquer, back-transformation,
occupations and mu, density matrix).

Metric: TFLOP/s of the fixed nominal count (36 M^3 per complex k-point + 4 M^2 n_rho for
the density matrix; 9 M^3 + M^2 n_rho for real problems), whole job over all ranks.
Inputs (8 x 709 MB per matrix) are far larger than L2, so no flush is needed.

--impl reference times the CPU oracle (the deliberately plain FP64 reference of this
project) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "kbatch512": dict(desc="512-atom Si supercell, N=6656, 8 k-points, complex128, shared mu", tiling=(4, 4, 4)),
    "kbatch64": dict(desc="64-atom Si supercell, N=832, 8 k-points, complex128, shared mu", tiling=(2, 2, 2)),
    "gamma64": dict(desc="64-atom Si cluster, N=832, Gamma, real", tiling=(2, 2, 2)),
    "nc384": dict(desc="384-atom Si cluster, noncollinear 2N=9984, complex128", tiling=(4, 4, 3)),
    "adjoint216": dict(desc="216-atom Si cluster, N=2808, Gamma, real", tiling=(3, 3, 3)),
    "product4096": dict(desc="one FP64-accurate split-bf16 product, complex 4096 x 4096 x 4096 (the tensor-core "
                             "kernel of the path on its own)", tiling=None),
    "uneven48": dict(desc="48 independent Si clusters of 16-160 atoms (N=208-2080), the first 12 noncollinear "
                          "(2N up to 4160, complex128), the rest real; one batched launch sequence", tiling=None),
}


def measured_fp64_peak(ctx, device):
    """The FP64 FMA pipe's throughput measured by the library's probe (gks_measure_peak),
    with the SM clock sampled while it ran; the FP64 roofline of a kernel timed at another
    clock scales it by the ratio of the clocks."""
    clk = ClockSampler(device)
    clk.start()
    dfma = ctx.measure_peak("dfma")
    dmma = ctx.measure_peak("dmma")
    c = clk.stop()
    return {"dfma_tflops": dfma, "dmma_tflops": dmma, "sm_mhz": c["sm_mhz"]}


def nominal_flops(M: int, complex_: bool, nrho) -> float:
    c = 36.0 if complex_ else 9.0
    r = 4.0 if complex_ else 1.0
    return sum(c * M ** 3 + r * M * M * float(n) for n in nrho)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def kshard_range(nk: int, world: int, rank: int):
    """Contiguous k-point range [k0, k1) of a rank: the k-points of one system spread as
    evenly as possible (the first nk % world ranks take one more)."""
    base, extra = divmod(nk, world)
    k0 = rank * base + min(rank, extra)
    return k0, k0 + base + (1 if rank < extra else 0)


def gather_eps(eps_local, nk: int, world: int):
    """All ranks' eigenvalues (nk, M) in k order from each rank's contiguous block (the one
    exchange of the k-point sharding: nk M doubles); ranks with fewer k-points pad."""
    import torch
    import torch.distributed as dist
    per = max(kshard_range(nk, world, r)[1] - kshard_range(nk, world, r)[0] for r in range(world))
    M = eps_local.shape[-1]
    buf = torch.zeros(per, M, dtype=eps_local.dtype, device=eps_local.device)
    buf[:eps_local.shape[0]] = eps_local
    out = torch.empty(world * per, M, dtype=eps_local.dtype, device=eps_local.device)
    dist.all_gather_into_tensor(out, buf)
    rows = []
    for r in range(world):
        k0, k1 = kshard_range(nk, world, r)
        rows.append(out[r * per:r * per + (k1 - k0)])
    return torch.cat(rows).contiguous()


def max_over_ranks(value: float, device) -> float:
    """The slowest rank's value (whole-job time); the value itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        return out


# ------------------------------------------------------------------ CPU oracle leg

SAMPLE_OF = {
    # one pencil of the same construction, sized for 10-30 s of the oracle on the host cores
    "kbatch512": ("216-atom (3,3,3) supercell, k-point 0 of the 2x2x2 mesh", "periodic", (3, 3, 3)),
    "kbatch64": ("64-atom (2,2,2) supercell, k-point 0", "periodic", (2, 2, 2)),
    "gamma64": ("the full 64-atom cluster", "cluster", (2, 2, 2)),
    "adjoint216": ("the full 216-atom (3,3,3) cluster", "cluster", (3, 3, 3)),
    "nc384": ("64-atom (2,2,1) noncollinear cluster", "nc", (2, 2, 1)),
    "uneven48": ("a 128-atom (4,2,2) real cluster of the batch's construction", "cluster", (4, 2, 2)),
}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OracleSampler:
    """The CPU oracle on one pencil of the workload's construction, in a child process
    (no CUDA) using every host core of the affinity mask; the pencil is built once."""

    def __init__(self, workload: str, seconds_cap: float = 900.0):
        self.workload = workload
        self.cap = seconds_cap
        self.cores = host_cores()
        self.dir = tempfile.mkdtemp(prefix="gks_oracle_sample_")
        desc, kind, tiling = SAMPLE_OF[workload]
        self.desc = desc
        code = f"""
import sys
sys.path.insert(0, {ROOT!r})
import numpy as np
from paper_2606_09058_gb300 import inputs as I
kind, tiling = {kind!r}, {tiling!r}
if kind == "periodic":
    p = I.periodic(tiling, 1, 0.01, 4.0 * 8 * tiling[0] * tiling[1] * tiling[2], kidx=[0])
elif kind == "nc":
    p = I.noncollinear(tiling, 2, 0.01)
else:
    p = I.collinear_gamma(tiling, 0, 0.01)
np.save({self.dir!r} + "/H.npy", p.H[:1].numpy()); np.save({self.dir!r} + "/S.npy", p.S[:1].numpy())
np.save({self.dir!r} + "/meta.npy", np.array([p.kT, p.n_elec, 1.0 if p.spin == "noncollinear" else 0.0]))
"""
        self._run(code)

    def _env(self):
        n = str(self.cores)
        return dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n, CUDA_VISIBLE_DEVICES="")

    def _run(self, code):
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=self._env(),
                           timeout=self.cap)
        if r.returncode != 0:
            raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
        return r.stdout

    def run(self) -> dict:
        code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import oracle as O
d = {self.dir!r}
H = np.load(d + "/H.npy"); S = np.load(d + "/S.npy"); kT, ne, nc = np.load(d + "/meta.npy")
t = time.perf_counter()
r = O.solve(H, S, kT, ne, "noncollinear" if nc else "collinear")
dt = time.perf_counter() - t
M = H.shape[1]; cplx = bool(np.iscomplexobj(H))
fl = (36.0 if cplx else 9.0) * M ** 3 + (4.0 if cplx else 1.0) * M * M * float(r.n_rho[0])
print(json.dumps(dict(seconds=dt, flops=fl, n=M, complex=cplx)))
"""
        res = json.loads(self._run(code).strip().splitlines()[-1])
        res["desc"] = self.desc
        res["cores"] = self.cores
        return res


def oracle_sample(workload: str, seconds_cap: float = 900.0) -> dict:
    return OracleSampler(workload, seconds_cap).run()


def _sample_text(workload, smp):
    return (f"one {smp['n']}x{smp['n']} {'complex' if smp['complex'] else 'real'} pencil of the same construction "
            f"({smp['desc']}) solved by the plain FP64 oracle (OpenMP, {smp['cores']} host cores) in "
            f"{smp['seconds']:.1f} s; rate of the nominal FP64 count")


def reference_arm(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    sampler = OracleSampler(args.workload)
    samples = []
    for _ in range(args.warmup + args.steps):
        samples.append(sampler.run())
    timed = samples[args.warmup:]
    secs = sum(s["seconds"] for s in timed)
    fl = sum(s["flops"] for s in timed)
    val = fl / secs / 1e12
    s0 = timed[0]
    cpu = {"value": val, "unit": "TFLOP/s", "cores": s0["cores"], "kind": "oracle",
           "sample": _sample_text(args.workload, s0)}
    line = {"impl": "reference", "metric": "GKS eigensolve+rho throughput (nominal FP64 TFLOP/s)", "value": val,
            "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample_n": s0["n"]},
            "cpu_baseline": cpu, "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

RESIDUE_MODULI = [256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193]


def split_products(form, Kp, bits=54):
    """bf16 products per split product: 45 digit pairs for nine 6-bit digits, or the number
    of moduli n of the residue form (the fewest with 2 Kp 2^{2p} <= prod m, p >= bits)."""
    if form == "digits":
        return 45
    M = 1
    for n, m in enumerate(RESIDUE_MODULI, 1):
        M *= m
        if min((M // (2 * Kp)).bit_length() - 1, 124) // 2 >= bits:
            return n
    return 45


def run_product(args):
    """One complex 4096^3 product through gks_gemm (split-bf16 products in the chosen form),
    with the tensor roofline of the executed bf16 work: per product 2 Mp N'p K'p bf16 flops
    for each bf16 product of the form (N' = 2N, K' = 2K for the real embedding)."""
    import numpy as np
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2606_09058_gb300 import build as B
    B.build()
    from paper_2606_09058_gb300 import gks
    n = 4096
    g = torch.Generator(device=dev).manual_seed(9058005)
    A = torch.randn(n, n, dtype=torch.complex128, device=dev, generator=g)
    Bm = torch.randn(n, n, dtype=torch.complex128, device=dev, generator=g)
    C = torch.zeros(n, n, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = gks.Context(local, stream, split=args.split)
    lib, h = ctx._lib, ctx._h

    def prod():
        rc = lib.gks_gemm(h, gks.GKS_C128, 0, 0, n, n, n, 1.0, A.data_ptr(), n, Bm.data_ptr(), n, 0.0, C.data_ptr(),
                          n, 2)
        if rc:
            raise RuntimeError(f"gks_gemm failed: {rc}")
    for _ in range(max(3, args.warmup)):
        prod()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = gks.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps = max(args.steps, 5)
    for _ in range(steps):
        prod()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = gks.launch_count() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    ref_err = None
    if rank == 0:  # spot check against torch's FP64 product on 64 rows
        ref = A[:64] @ Bm
        ref_err = float(((C[:64] - ref).abs().max() / ref.abs().max()).item())
    fl = 8.0 * n ** 3
    nprod = split_products(args.split, 2 * n)
    bf16 = 2.0 * n * (2 * n) * (2 * n) * nprod
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    ach = bf16 / (ms / 1e3) / 1e12
    if rank == 0:
        line = {"metric": "FP64-accurate complex product throughput (FP64-equivalent TFLOP/s)",
                "value": fl / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "n_gpus": 1, "steps": steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16 split values, fp32 tensor accumulation", "data": "synthetic",
                "config": {"workload": "product4096", "desc": WORKLOADS["product4096"]["desc"],
                           "split_form": args.split, "bf16_products": nprod,
                           "max_rel_err_vs_fp64_rows0_63": ref_err,
                           "l2": "operands and digits (1.8 GB) larger than L2 (no flush needed)"},
                "roofline": {"bound": "tensor", "achieved": ach, "peak": bf16_peak, "unit": "TFLOP/s",
                             "frac": ach / bf16_peak, "traffic": None,
                             "kernel": ("crt_tc_kernel + oz_split_kernel + crt_recon_kernel" if args.split == "residues"
                                        else "oz_tc_kernel + oz_split_kernel"),
                             "peak_basis": "bf16 dense, MEASURED_PEAKS.json burst"},
                "cpu_baseline": None, "e2e": None, "gpu_launches": int(launches),
                "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}}
        print(json.dumps(line), flush=True)
    return 0


def run_uneven(args):
    """48 independent systems of uneven order in one batched launch sequence per step
    (gks_solve_batched), after tuning the outer width per shape class (not timed)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from math import exp

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        from paper_2606_09058_gb300 import build as B
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2606_09058_gb300 import gks, inputs as I

    probs = I.uneven_batch(device=str(dev))
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)  # the batched solve forks its worker streams from a non-default stream
    ctx = gks.Context(local, stream, graph=not args.no_graph, precision=args.precision, split=args.split,
                      hemv=args.hemv)
    tuned = {}
    if not args.no_tune:
        seen = set()
        for p in probs:
            n, cplx = p.S.shape[-1], p.H.is_complex()
            M = p.H.shape[-1]
            b = 1 << max(6, (M - 1).bit_length())
            key = (b, cplx, p.spin)
            if key in seen:
                continue
            seen.add(key)
            best, _ = ctx.tune(n, 1, cplx, p.spin, widths=(64, 128, 256))
            tuned[f"{'nc' if p.spin == 'noncollinear' else ('c' if cplx else 'r')}{b}"] = best
    items = [dict(H=p.H.contiguous(), S=p.S.contiguous(), kT=p.kT, n_elec=p.n_elec, spin=p.spin) for p in probs]
    sols = None
    per_pass = 0
    for w in range(max(2, args.warmup)):  # eager, then capture (graph mode), then replays
        c0 = gks.launch_count()
        sols = ctx.solve_batched(items, nstreams=8, sync=True, out=sols)
        if w == 0:
            per_pass = gks.launch_count() - c0  # kernels of one eager pass (what a replay runs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = gks.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.solve_batched(items, nstreams=8, sync=False, out=sols)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = gks.launch_count() - l0
    if launches == 0 and not args.no_graph:
        launches = per_pass * args.steps  # graph replays launch the captured kernels without the host
    clk = clocks.stop()
    ctx.sync()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)

    def fermi(x):
        return exp(-x) / (1 + exp(-x)) if x > 0 else 1 / (1 + exp(x))
    fl = 0.0
    for p, sol in zip(probs, sols):
        M = p.H.shape[-1]
        e = sol.eps.cpu().numpy()[0]
        m = float(sol.mu.item())
        nr = sum(1 for v in e if fermi((v - m) / p.kT) >= 1e-16)
        fl += nominal_flops(M, p.H.is_complex(), [nr])
    value = fl * world / (ms / 1e3) / 1e12
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            smp = oracle_sample(args.workload)
            cpu = {"value": smp["flops"] / smp["seconds"] / 1e12, "unit": "TFLOP/s", "cores": smp["cores"],
                   "kind": "oracle", "sample": _sample_text(args.workload, smp)}
        except Exception as ex:
            cpu = {"value": None, "unit": "TFLOP/s", "cores": host_cores(), "kind": "oracle",
                   "sample": f"failed: {ex}"[:300]}
    if rank == 0:
        line = {"metric": "GKS eigensolve+rho throughput (nominal FP64 TFLOP/s)", "value": value, "unit": "TFLOP/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "systems": len(probs),
                           "systems_per_s": len(probs) * world / (ms / 1e3), "precision": args.precision,
                           "graph": not args.no_graph,
                           "gpu_launches_counted": ("kernels of one eager pass x graph replays" if not args.no_graph
                                                    else "host launches in the timed region"),
                           "tuned_widths": tuned, "nominal_tflop_per_step": fl / 1e12,
                           "l2": "48 systems, 2.4 GB of inputs, larger than L2 (no flush needed)"},
                "roofline": None, "cpu_baseline": cpu, "e2e": None, "gpu_launches": int(launches),
                "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def accuracy_report(workload, prob, H, S, eps, C, mu, nrho):
    """Accuracy of the timed step's results: eigenvalues of every k-point against the oracle's
    (tests/golden/kbatch512_oracle.npz holds k-points 0..3; k and -k share a spectrum), over
    the occupied states (f >= 1e-16) and over all states, against the gate max(1e-10, 8 beta_i);
    scaled S-orthonormality and backward error of every column of k-point 0 (FP64 products
    in torch); Tr(rho S) is checked by the tests.  None for workloads without stored results."""
    import numpy as np
    import torch
    out = {}
    gpath = os.path.join(ROOT, "tests", "golden", f"{workload}_oracle.npz")
    if workload == "kbatch512" and os.path.exists(gpath):
        g = np.load(gpath)
        e = eps.cpu().numpy()
        worst_occ = worst_all = ratio = 0.0
        nbig = 0
        for k in range(e.shape[0]):
            r = k if k < 4 else 7 - k
            if f"eps{r}" not in g.files:
                continue
            d = np.abs(e[k] - g[f"eps{r}"])
            gate = np.maximum(1e-10, 8 * g[f"beta{r}"])
            worst_occ = max(worst_occ, float(d[:nrho[k]].max()))
            worst_all = max(worst_all, float(d.max()))
            ratio = max(ratio, float((d / gate).max()))
            nbig += int(np.sum(g[f"beta{r}"][:nrho[k]] > 1e-11))
        out.update({"max_abs_deps_occupied": worst_occ, "max_abs_deps_all": worst_all,
                    "max_deps_over_gate": ratio,
                    "gate": "max(1e-10, 8 beta_i), beta_i = u (|H| + |eps_i| |S|) |c_i|^2",
                    "occupied_states_with_beta_above_1e-11": nbig,
                    "reference": "oracle eigenvalues of the same pencils (tests/golden/kbatch512_oracle.npz)"})
    if C.shape[1] != C.shape[2]:
        return out or None
    k = 0
    Hk, Sk, Ck, ek = H[k], S[k], C[k], eps[k]
    if Hk.shape[0] != Sk.shape[0]:  # noncollinear: S_NC = I_2 (x) S
        n = Sk.shape[0]
        Sn = torch.zeros(2 * n, 2 * n, dtype=Sk.dtype, device=Sk.device)
        Sn[:n, :n] = Sk
        Sn[n:, n:] = Sk
        Sk = Sn
    def norm2(A, iters=100):
        v = torch.ones(A.shape[0], dtype=A.dtype, device=A.device) / A.shape[0] ** 0.5
        lam = 0.0
        for _ in range(iters):
            w = A @ v
            lam = float(torch.linalg.norm(w))
            v = w / lam
        return lam
    nh, ns = norm2(Hk), norm2(Sk)
    cn = torch.linalg.norm(Ck, dim=0)
    SC = Sk @ Ck
    G = Ck.conj().T @ SC
    G.diagonal().sub_(1.0)
    out["orthonormality_scaled_k0"] = float((G.abs() / torch.outer(cn, cn)).max()) / ns
    del G
    R = Hk @ Ck - SC * ek[None, :]
    out["backward_error_scaled_k0"] = float((torch.linalg.norm(R, dim=0) / ((nh + ek.abs() * ns) * cn)).max())
    out["orthonormality_gate"] = 1e-12 * Ck.shape[0] ** 0.5
    del R, SC
    return out


def make_problem(workload: str, device: str):
    from paper_2606_09058_gb300 import inputs as I
    return I.workload(workload, device=device)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kbatch512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the mixed-precision and one-problem-per-call forms of the step")
    ap.add_argument("--profile-json", default=None, help="write the per-class/per-stage event profile here")
    ap.add_argument("--no-tune", action="store_true", help="uneven48: skip the width tuner")
    ap.add_argument("--no-graph", action="store_true", help="uneven48: eager launches instead of graph replay")
    ap.add_argument("--gemm", default="auto", choices=["auto", "fp64", "split"],
                    help="products: auto (split-bf16 tensor-core products where they pay), fp64 (FP64 pipe only)")
    ap.add_argument("--block", type=int, default=0, help="outer block width (0 = library default)")
    ap.add_argument("--tridiag", default="one_stage", choices=["one_stage", "two_stage"],
                    help="tridiagonalization of the timed step")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"], help="arithmetic of the timed step")
    ap.add_argument("--split", default="residues", choices=["residues", "digits"],
                    help="form of the FP64-accurate tensor-core products")
    ap.add_argument("--hemv", default="digits", choices=["digits", "fp64"],
                    help="form of the one-stage matrix-vector step")
    ap.add_argument("--per-k", action="store_true",
                    help="solve the k-points one call each (nk = 1, shared mu lost) instead of one batched call")
    ap.add_argument("--k-points", type=int, default=0,
                    help="keep only the first N k-points of the workload (a small case for kernel captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "uneven48":
        return run_uneven(args)
    if args.workload == "product4096":
        return run_product(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        from paper_2606_09058_gb300 import build as B
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2606_09058_gb300 import gks

    # Under torchrun the k-points of the one system are sharded: rank r owns a contiguous
    # k range, solves it (eigenpairs only), the eigenvalues of all k-points are allgathered
    # (NCCL, nk M doubles) and every rank runs the same bisection for the shared mu
    # (gks_occupy) before its own density matrices: strong scaling of one system.  A
    # workload with fewer k-points than ranks runs replicas (weak scaling).
    prob = make_problem(args.workload, str(dev))
    if 0 < args.k_points < prob.H.shape[0]:
        n_keep = args.k_points
        prob.H, prob.S = prob.H[:n_keep].contiguous(), prob.S[:n_keep].contiguous()
        prob.kweights = np.full(n_keep, 1.0 / n_keep)
        prob.nk = n_keep
        torch.cuda.empty_cache()
    nk_all = prob.H.shape[0]
    shard = world > 1 and nk_all >= world and prob.spin == "collinear" and not args.per_k
    k0, k1 = kshard_range(nk_all, world, rank) if shard else (0, nk_all)
    H, S = prob.H[k0:k1].contiguous(), prob.S[k0:k1].contiguous()
    if shard:
        del prob.H, prob.S
    nk, M = H.shape[0], H.shape[1]
    spin = prob.spin
    kw = torch.as_tensor(np.asarray(prob.kweights, float), device=dev)  # all k-points (1/nk_all)
    kw_local = kw[k0:k1].contiguous()
    stream = torch.cuda.current_stream(dev)
    ctx = gks.Context(local, stream, profile=True, gemm=args.gemm, block=args.block, tridiag=args.tridiag,
                      precision=args.precision, split=args.split, hemv=args.hemv)
    eps = torch.empty(nk, M, dtype=torch.float64, device=dev)
    C = torch.empty(nk, M, M, dtype=H.dtype, device=dev)
    rho = torch.empty_like(C)
    mu = torch.empty(1, dtype=torch.float64, device=dev)
    eb = torch.empty(1, dtype=torch.float64, device=dev)

    # the differentiation workload: one step is the forward solve plus the adjoint of a loss with
    # a seeded Hermitian density-matrix cotangent and the band energy
    adj = args.workload == "adjoint216" and not shard
    rbar = None
    if adj:
        gen = torch.Generator(device=dev).manual_seed(9058004)
        rbar = torch.randn(nk, M, M, generator=gen, device=dev, dtype=torch.float64)
        if H.is_complex():
            rbar = torch.complex(rbar, torch.randn(nk, M, M, generator=gen, device=dev, dtype=torch.float64))
        rbar = 0.5 * (rbar + rbar.transpose(-1, -2).conj())

    def step(Hd, Sd, sync=False):
        if adj:
            ctx.solve_into(Hd, Sd, prob.kT, prob.n_elec, spin, kw, eps=eps, C=C, mu=mu, rho=rho, e_band=eb,
                           sync=False, save_for_backward=True)
            ctx.adjoint(None, Sd, prob.kT, spin, kw, rho_bar=rbar, e_band_bar=1.0, sync=sync,
                        complex_=H.is_complex())
            return
        if args.per_k:  # one problem per call: the per-problem baseline for the batched form
            for k in range(nk):
                ctx.solve_into(Hd[k:k + 1], Sd[k:k + 1], prob.kT, prob.n_elec, spin, None,
                               eps=eps[k:k + 1], C=C[k:k + 1], mu=mu, rho=rho[k:k + 1], e_band=eb, sync=sync)
            return
        if shard:
            ctx.solve_into(Hd, Sd, prob.kT, prob.n_elec, spin, kw_local, eps=eps, C=C, sync=False, eigen_only=True)
            eps_all = gather_eps(eps, nk_all, world)
            m_, r_, e_, _ = ctx.occupy(eps_all, C, prob.kT, prob.n_elec, k0=k0, spin=spin, kweights_all=kw,
                                       sync=sync)
            mu.copy_(m_)
            rho.copy_(r_)
            eb.copy_(e_)
            return
        ctx.solve_into(Hd, Sd, prob.kT, prob.n_elec, spin, kw, eps=eps, C=C, mu=mu, rho=rho, e_band=eb, sync=sync)

    for _ in range(args.warmup):
        step(H, S, sync=True)
    ctx.profile()  # drop warm-up records
    peak = measured_fp64_peak(ctx, local)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = gks.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step(H, S)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = gks.launch_count() - l0
    clk = clocks.stop()
    ctx.sync()
    prof = ctx.profile()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)

    eps_h = eps.cpu().numpy()
    mu_h = float(mu.item())
    from math import exp

    def fermi(x):
        return exp(-x) / (1 + exp(-x)) if x > 0 else 1 / (1 + exp(x))
    nrho = [int(sum(1 for v in eps_h[k] if fermi((v - mu_h) / prob.kT) >= 1e-16)) for k in range(nk)]
    fl_step = nominal_flops(M, H.is_complex(), nrho)
    if adj:
        # the adjoint: six M x M x M products per item (C^H rho_bar C, C B_H C^H, C B_S C^H)
        fl_step += (48.0 if H.is_complex() else 12.0) * M ** 3 * nk
    if shard:  # strong scaling: the k-points of one system over the ranks
        ft = torch.tensor([fl_step], dtype=torch.float64, device=dev)
        dist.all_reduce(ft)
        fl_job = float(ft.item())
    else:      # replicas (weak scaling): every rank solves the whole workload
        fl_job = fl_step * world
    value = fl_job / (ms / 1e3) / 1e12

    # roofline: dominant kernel class over the timed region.  DRAM traffic per launch comes
    # from one ncu capture of the kernel on the 64-atom k-batch (profiles/), where it matched
    # the algorithmic bytes of that launch to the ratio below; it scales with the bytes the
    # launch processes, so the live per-launch algorithmic bytes times that ratio is reported.
    # DRAM bytes / algorithmic bytes of one launch from an ncu capture (profiles/) of the
    # kernel as it stands: the FP64 matrix-vector step (16-row blocks on the 64-atom k-batch)
    # and its digit form (one k-point of the 512-atom batch, the tiled copy-ring version:
    # DRAM bytes = the digit block)
    TRAFFIC_RATIO = {("hetrd_hemv", "fp64"): 1.04, ("hetrd_hemv", "digits"): 1.019}
    kern = [p for p in prof if not p["name"].startswith("stage:")]
    dom = max(kern, key=lambda p: p["ms"]) if kern else None
    roof = None
    if dom:
        per = args.steps
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12 if dom["ms"] > 0 else 0.0
        scale = (clk["sm_mhz"] / peak["sm_mhz"]) if (clk["sm_mhz"] and peak["sm_mhz"]) else 1.0
        pk = peak["dfma_tflops"] * scale
        form = args.hemv if dom["name"] == "hetrd_hemv" and args.precision == "fp64" else "fp64"
        ratio = TRAFFIC_RATIO.get((dom["name"], form))
        traffic = ratio * dom["bytes"] / dom["groups"] if ratio and dom.get("groups") else None
        fp64_eq = {"achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                   "peak_basis": (f"FP64 DFMA pipe measured by gks_measure_peak in this run: "
                                  f"{peak['dfma_tflops']:.3f} TFLOP/s at {peak['sm_mhz']} MHz, scaled to the "
                                  f"timed region's median SM clock (DMMA measured {peak['dmma_tflops']:.3f})")}
        common = {"traffic": traffic, "kernel": dom["name"], "kernel_ms_per_step": dom["ms"] / per,
                  "kernel_share": dom["ms"] / (ms * per)}
        if dom["name"] == "split_gemm":
            # the tensor-core products: every bf16 product of the split form executes the
            # nominal flops of the FP64 product (the complex embedding included), 16 of them
            # for the residue form (16 moduli), 45 for nine-digit pairs; against the
            # sustained bf16 peak (the kernels run inside a long step)
            nprod = 16 if args.split == "residues" else 45
            try:
                pk_t = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
                bf = float(pk_t["bf16_tflops_sustained"])
                basis = "bf16 dense sustained, MEASURED_PEAKS.json"
            except (OSError, KeyError, ValueError):
                bf, basis = 1700.0, "fallback 1.7 PFLOP/s sustained"
            ex = achieved * nprod
            roof = {"bound": "tensor", "achieved": ex, "peak": bf, "unit": "TFLOP/s", "frac": ex / bf, **common,
                    "peak_basis": basis,
                    "executed_per_nominal": nprod,
                    "note": ("executed bf16 work = nominal FP64 flops x bf16 products per product; the class "
                             "includes the splitting and reconstruction kernels"),
                    "fp64_equivalent": fp64_eq}
        elif form == "digits":
            # the digit form reads its digit block once per step: bytes / time against the
            # measured HBM copy rate (burst: the kernel runs inside a long step, but it is
            # memory-bound, where the copy rate is the ceiling)
            try:
                hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
                basis = "HBM copy rate, MEASURED_PEAKS.json"
            except (OSError, KeyError, ValueError):
                hbm, basis = 6800.0, "fallback 6.8 TB/s"
            gbs = dom["bytes"] / (dom["ms"] / 1e3) / 1e9 if dom["ms"] > 0 else 0.0
            roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, **common,
                    "peak_basis": basis, "fp64_equivalent": fp64_eq}
        else:
            roof = {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                    **common, "peak_basis": fp64_eq["peak_basis"]}
    stages = {p["name"][6:]: round(p["ms"] / args.steps, 3) for p in prof if p["name"].startswith("stage:")}
    classes = {p["name"]: {"ms": round(p["ms"] / args.steps, 3),
                           "tflops": round(p["flops"] / (p["ms"] / 1e3) / 1e12, 4) if p["ms"] > 0 and p["flops"] > 0
                           else None} for p in kern}
    if args.profile_json and rank == 0:
        with open(args.profile_json, "w") as fh:
            json.dump({"ms_per_step": ms, "profile": prof, "steps": args.steps}, fh, indent=1)

    # the other forms of the same step on the same GPU: mixed precision + refinement, and the
    # plain FP64 path one problem (k-point) per call
    compare = None
    if (not args.no_compare and not args.per_k and args.gemm == "auto" and world == 1 and args.tridiag == "one_stage"
            and args.precision == "fp64"):
        compare = {}

        def timed(fn, steps):
            fn()
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(steps):
                fn()
            a1.record(stream)
            torch.cuda.synchronize()
            return a0.elapsed_time(a1) / steps
        if M <= 18000:
            cm = gks.Context(local, stream, precision="mixed", block=args.block, split=args.split, hemv=args.hemv)
            eps_m = torch.empty_like(eps)
            C_m = torch.empty_like(C)
            rho_m = torch.empty_like(rho)
            mu_m = torch.empty_like(mu)
            eb_m = torch.empty_like(eb)
            mms = timed(lambda: cm.solve_into(H, S, prob.kT, prob.n_elec, spin, kw, eps=eps_m, C=C_m, mu=mu_m,
                                              rho=rho_m, e_band=eb_m, sync=False), args.steps)
            cm.sync()
            st = cm.refine_stats()
            nrho_m = [int(sum(1 for v in eps_m.cpu().numpy()[k] if fermi((v - float(mu_m.item())) / prob.kT) >= 1e-16))
                      for k in range(nk)]
            compare["mixed"] = {
                "ms_per_step": mms, "value": fl_step * world / (mms / 1e3) / 1e12, "unit": "TFLOP/s",
                "speedup_vs_fp64": ms / mms, "refine_sweeps": int(st.shape[0] // max(1, nk)),
                "refine_orthonormality_defect_per_sweep": [float(x) for x in st[:, 0].reshape(-1, nk).max(axis=1)],
                "abs_dmu_vs_fp64": abs(float(mu_m.item()) - mu_h),
                "accuracy": accuracy_report(args.workload, prob, H, S, eps_m, C_m, float(mu_m.item()), nrho_m)
                if not args.no_accuracy else None}
            del cm, eps_m, C_m, rho_m
            torch.cuda.empty_cache()
        # the other split-product form; two-stage tridiagonalization, all eigenvectors and the
        # lowest n_ev (occupied + margin)
        n_ev = min(M, max(nrho) + 64)
        other = "digits" if args.split == "residues" else "residues"
        other_hemv = "fp64" if args.hemv == "digits" else "digits"
        for name, kw_ in ((f"split_{other}", dict(split=other, hemv=args.hemv)),
                          (f"hemv_{other_hemv}", dict(split=args.split, hemv=other_hemv)),
                          ("two_stage", dict(tridiag="two_stage", split=args.split)),
                          ("one_stage_partial", dict(n_ev=n_ev, split=args.split, hemv=args.hemv)),
                          ("two_stage_partial", dict(tridiag="two_stage", n_ev=n_ev, split=args.split))):
            try:
                cx = gks.Context(local, stream, block=args.block, **kw_)
                ncol = kw_.get("n_ev", M)
                Cx = torch.empty(nk, M, ncol, dtype=H.dtype, device=dev)
                ex, rx = torch.empty_like(eps), torch.empty_like(rho)
                mx, bx = torch.empty_like(mu), torch.empty_like(eb)
                tms = timed(lambda: cx.solve_into(H, S, prob.kT, prob.n_elec, spin, kw, eps=ex, C=Cx, mu=mx, rho=rx,
                                                  e_band=bx, sync=False), args.steps)
                cx.sync()
                drho = float((rx - rho).abs().max()) / max(1e-300, float(rho.abs().max()))
                compare[name] = {"ms_per_step": tms, "speedup_vs_fp64_one_stage": ms / tms,
                                 "n_ev": ncol, "max_abs_deps_vs_fp64": float((ex - eps).abs().max()),
                                 "max_rel_drho_vs_fp64": drho}
                del cx, Cx, ex, rx
                torch.cuda.empty_cache()
            except Exception as ex_:  # a comparison form must not hide the main result
                compare[name] = {"error": str(ex_)[:300]}
        if nk > 1:
            saved = args.per_k
            args.per_k = True
            pms = timed(lambda: step(H, S), 1)
            args.per_k = saved
            ctx.sync()
            compare["fp64_per_problem"] = {"ms_per_step": pms, "value": fl_step * world / (pms / 1e3) / 1e12,
                                           "unit": "TFLOP/s", "batched_speedup": pms / ms,
                                           "note": "one gks_solve per k-point (nk = 1 each, 1 timed step)"}
        ctx.profile()

    # end to end through the C ABI with host buffers (pinned), H2D and D2H inside the timed region
    e2e = None
    if not args.no_e2e:
        Hh = torch.empty(H.shape, dtype=H.dtype, pin_memory=True)
        Sh = torch.empty(S.shape, dtype=S.dtype, pin_memory=True)
        Hh.copy_(H)
        Sh.copy_(S)
        eps_out = torch.empty(eps.shape, dtype=eps.dtype, pin_memory=True)
        mu_out = torch.empty(1, dtype=torch.float64, pin_memory=True)
        eb_out = torch.empty(1, dtype=torch.float64, pin_memory=True)
        C_out = torch.empty(C.shape, dtype=C.dtype, pin_memory=True)
        rho_out = torch.empty(rho.shape, dtype=rho.dtype, pin_memory=True)
        Hd = torch.empty_like(H)
        Sd = torch.empty_like(S)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            Hd.copy_(Hh, non_blocking=True)
            Sd.copy_(Sh, non_blocking=True)
            step(Hd, Sd)
            eps_out.copy_(eps, non_blocking=True)
            mu_out.copy_(mu, non_blocking=True)
            eb_out.copy_(eb, non_blocking=True)
            C_out.copy_(C, non_blocking=True)
            rho_out.copy_(rho, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        ctx.sync()
        ctx.profile()
        ems = max_over_ranks(f0.elapsed_time(f1) / args.steps, dev)
        e2e = {"value": fl_job / (ems / 1e3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(Hh.numel() * Hh.element_size() + Sh.numel() * Sh.element_size()),
               "d2h_bytes_per_step": int(eps_out.numel() * 8 + 16 + C_out.numel() * C_out.element_size()
                                         + rho_out.numel() * rho_out.element_size()),
               "ms_per_step": ems, "outputs_copied": "eps, mu, E_band, C, rho to pinned host memory"}
        del Hh, Sh, Hd, Sd, C_out, rho_out

    accuracy = None
    if world == 1 and not args.no_accuracy:
        accuracy = accuracy_report(args.workload, prob, H, S, eps, C, mu_h, nrho)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            del C, rho
            torch.cuda.empty_cache()
            smp = oracle_sample(args.workload)
            cpu = {"value": smp["flops"] / smp["seconds"] / 1e12, "unit": "TFLOP/s", "cores": smp["cores"],
                   "kind": "oracle", "sample": _sample_text(args.workload, smp)}
        except Exception as ex:  # the CPU leg must not hide the GPU result
            cpu = {"value": None, "unit": "TFLOP/s", "cores": host_cores(), "kind": "oracle",
                   "sample": f"failed: {ex}"[:300]}

    if rank == 0:
        line = {"metric": "GKS eigensolve+rho throughput (nominal FP64 TFLOP/s)", "value": value, "unit": "TFLOP/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong" if shard else "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "M": M, "nk": nk_all,
                           "parallelism": (f"k-point shard over {world} ranks (contiguous k ranges, allgather of "
                                           f"eps, shared mu on every rank)") if shard else
                           (f"{world} replicas" if world > 1 else "one GPU"),
                           "spin": spin, "precision": args.precision, "tridiag": args.tridiag,
                           "products": args.gemm, "split_form": args.split, "hemv_form": args.hemv,
                           "block": args.block or (512 if M >= 4096 else 256),
                           "batching": "one call per k-point" if args.per_k else "all k-points in one call",
                           "l2": "inputs larger than L2 (no flush needed)",
                           "nominal_tflop_per_step": fl_step / 1e12, "n_rho": nrho},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
                "accuracy": accuracy, "compare": compare, "fp64_peaks_measured": peak,
                "stages_ms": stages, "kernels": classes}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
