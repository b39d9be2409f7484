"""Host-side pieces of bench.py: the exact update count U behind the metric, and
the JSON line of the reference (oracle) arm."""
import json
import os
import subprocess
import sys

import numpy as np

import oracle
import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _brute_force_updates(norb, na, nb, x):
    """sum_k #{t in S : t ^ x_k in S} by enumerating the sector."""
    s = oracle.Sector.molecular(norb, na, nb)
    cfg = s.configs().astype(np.uint64)
    lo = np.uint64((1 << norb) - 1)

    def in_sector(b):
        pa = np.array([bin(int(v)).count("1") for v in (b & lo)])
        pb = np.array([bin(int(v)).count("1") for v in (b >> np.uint64(norb))])
        return (pa == na) & (pb == nb)

    total = 0
    for xv in np.unique(x):
        cnt = int(np.count_nonzero(x == xv))
        total += cnt * int(np.count_nonzero(in_sector(cfg ^ np.uint64(xv))))
    return total


def test_update_count_matches_enumeration():
    sys.path.insert(0, ROOT)
    from bench import count_updates
    for norb, na, nb, seed in [(6, 3, 3, 0), (6, 2, 3, 1), (8, 4, 4, 2)]:
        h, g = w.molecular_integrals(norb, seed)
        H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
        x = np.asarray(H.x, dtype=np.uint64)
        assert count_updates(x, norb, norb, na, nb) == _brute_force_updates(norb, na, nb, x)
        # the group-level count U_g behind the gather rate: one source read per
        # (target, group) pair with a contribution
        xg = np.unique(x)
        assert count_updates(xg, norb, norb, na, nb) == _brute_force_updates(norb, na, nb, xg)


def test_update_counts_of_the_12_qubit_molecule():
    """6 orbitals, (3a,3b), D = 400: U = 400 * 907 term updates and U_g = 400 * 118
    group updates (907 terms and 118 groups with a source in the sector per target on
    average), the counts behind the metric and the gather rate."""
    sys.path.insert(0, ROOT)
    from bench import count_updates
    h, g = w.MOL12.integrals()
    H = oracle.jw_hamiltonian(6, h, g, eps_drop=1e-12)
    x = np.asarray(H.x, dtype=np.uint64)
    assert count_updates(x, 6, 6, 3, 3) == 400 * 907
    assert count_updates(np.unique(x), 6, 6, 3, 3) == 400 * 118


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-seconds", "0.5"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from bench import max_over_ranks
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        q.put((rank, max_over_ranks(1.5 + rank, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_step_time_is_the_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_reference_arm_under_torchrun_prints_one_line():
    """Two ranks: rank 0 alone runs the oracle and prints; rank 1 exits 0 at once."""
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-seconds",
                        "0.3"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
