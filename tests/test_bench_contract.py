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
