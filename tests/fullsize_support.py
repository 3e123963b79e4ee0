"""Inputs and oracle results for the parity test of the 48 uneven systems at their own sizes.

The oracle needs minutes for the whole batch on the host cores, so the GPU test session
starts it early: at the end of collection, when the full-size tests are selected and a
CUDA device is present, `start()` builds the 48 pencils on the device (the same arrays the
CUDA path will solve), writes them to a scratch directory and launches `oracle_job.py` on
them in a separate process (a fresh interpreter, so no CUDA state is shared).  The test,
collected late, waits for its results with `oracle_result()`.  Nothing here computes an
expected value: the job calls only oracle/.  (The 512-atom and 384-atom results, hours of
oracle time, are stored under tests/golden/ by make_fullsize.py.)
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

_state: dict = {}


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def start() -> None:
    """Build the full-size inputs on cuda:0 and start the oracle job (idempotent)."""
    if _state.get("started"):
        return
    _state["started"] = True
    import torch
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2606_09058_gb300 import inputs as I
    d = tempfile.mkdtemp(prefix="gks_fullsize_")
    _state["dir"] = d
    t0 = time.time()
    probs = I.uneven_batch(device="cuda")
    _state["uneven48"] = probs
    for b, p in enumerate(probs):
        np.save(os.path.join(d, f"u{b}_H.npy"), p.H[0].cpu().numpy())
        np.save(os.path.join(d, f"u{b}_S.npy"), p.S[0].cpu().numpy())
    meta = {"u": [(p.kT, p.n_elec, p.spin) for p in probs]}
    np.save(os.path.join(d, "meta.npy"), np.array(meta, dtype=object), allow_pickle=True)
    _state["gen_s"] = time.time() - t0
    n = str(cores())
    env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n, CUDA_VISIBLE_DEVICES="")
    log = open(os.path.join(d, "job.log"), "w")
    _state["proc"] = subprocess.Popen([sys.executable, os.path.join(HERE, "oracle_job.py"), d], env=env,
                                      stdout=log, stderr=subprocess.STDOUT, cwd=ROOT)


def started() -> bool:
    return bool(_state.get("started")) and "proc" in _state


def inputs(name: str):
    return _state[name]


def oracle_result(name: str, timeout: float = 1500.0) -> dict:
    """Wait for `<name>.npz` of the oracle job (raises if the job failed or timed out)."""
    d = _state["dir"]
    path = os.path.join(d, name + ".npz")
    t0 = time.time()
    while not os.path.exists(path):
        if _state["proc"].poll() is not None and not os.path.exists(path):
            raise RuntimeError("oracle job ended without " + name + ": " + open(os.path.join(d, "job.log")).read()[-2000:])
        if time.time() - t0 > timeout:
            raise TimeoutError("oracle job did not produce " + name)
        time.sleep(2.0)
    with np.load(path, allow_pickle=True) as z:
        return {k: z[k] for k in z.files}


def stop() -> None:
    p = _state.get("proc")
    if p is not None and p.poll() is None:
        p.kill()
        p.wait()
