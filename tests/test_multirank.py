"""The N > 1 host path on the CPU (gloo, world size 2): whole-job time is the slowest rank's,
and under torchrun only rank 0 prints the benchmark line (the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    out[rank] = bench.max_over_ranks(1.5 + rank, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == 2.5 and out[1] == 2.5


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload",
                        "gamma64"], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_kshard_ranges_partition_the_kpoints():
    sys.path.insert(0, ROOT)
    import bench
    for nk in (1, 2, 7, 8, 9):
        for world in range(1, nk + 1):
            seen = []
            for r in range(world):
                k0, k1 = bench.kshard_range(nk, world, r)
                assert 0 <= k0 <= k1 <= nk and k1 - k0 in (nk // world, nk // world + 1)
                seen.extend(range(k0, k1))
            assert seen == list(range(nk))


def _kshard_worker(rank, world, port, out):
    """Each rank solves its contiguous k range with the oracle, the eigenvalues are gathered
    in k order over gloo (the one exchange of the k-point shard), and every rank runs the
    same bisection: mu and E_band equal the single-process oracle's bit for bit."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from oracle import oracle as O
    from paper_2606_09058_gb300 import inputs as I
    p = I.periodic((1, 1, 1), 1, 0.01)
    nk = p.nk
    k0, k1 = bench.kshard_range(nk, world, rank)
    eps_local = torch.as_tensor(np.stack([O.eigh_generalized(p.H[k].numpy(), p.S[k].numpy())[0]
                                          for k in range(k0, k1)]))
    eps_all = bench.gather_eps(eps_local, nk, world).numpy()
    w = np.asarray(p.kweights, float)
    mu = O.chemical_potential(eps_all, w, 2.0, p.kT, p.n_elec)
    out[rank] = (mu, eps_all.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_kshard_gather_and_shared_mu_gloo_two_ranks():
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import oracle as O
    from paper_2606_09058_gb300 import inputs as I
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_kshard_worker, args=(2, port, out), nprocs=2, join=True)
    p = I.periodic((1, 1, 1), 1, 0.01)
    ref = O.solve(p.H.numpy(), p.S.numpy(), p.kT, p.n_elec, kweights=p.kweights)
    for r in range(2):
        mu, eb = out[r]
        assert mu == ref.mu
        assert eb == np.ascontiguousarray(ref.eps).tobytes()
