"""Potential-energy scan with the pair-double ansatz: previous-point start vs
the learned warm start (Sec. 4).

    python -m paper_2606_28952_gb300.pes_scan --norb 8 --points 40 --dtype c128

Both arms optimise the same ansatz at the same points R (h(R) = h0 + R h1,
g(R) = g0 exp(-0.3 R), seeded synthetic integrals) with the same L-BFGS
settings.  The previous-point arm starts every point from the angles the
previous point converged to; the learned arm starts from the network's
predicted move theta_prev + f(R) - f(R_prev) once the network has seen
`min_train` points, if that start has the lower energy of the two (two
energy-only evaluations per point, counted; otherwise it falls back to the
previous angles).  The first `min_train` points are the same in both arms and
are computed once.  Per point, E_ref = the lower of the two
converged energies, and each arm reports the L-BFGS iterations, energy /
gradient evaluations and wall time until its energy first came within
1e-6 Ha of E_ref.  Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import PauliSum, Sector
from .vqe import EnergyGradient, ProductAnsatz, WarmStart, iterations_to, scan

TARGET = 1e-6


def seniority_rows(S: Sector, norb: int):
    """Sector indices of the seniority-zero configurations (device int64): the
    pair-double ansatz maps them onto themselves and the closed-shell
    reference is one of them."""
    import torch
    import workloads as w
    cfg = w.seniority_zero_configs(norb, norb // 2).astype(np.int64)
    rows = S.rank(torch.from_numpy(cfg).cuda())
    if int((rows < 0).sum().item()) != 0:
        raise ValueError("a seniority-zero configuration is outside the sector")
    return rows


def make_scan_problem(norb: int, count: int, dtype, seed: int, support: bool = False):
    import workloads as w
    h0, h1, g0 = w.pes_integrals(norb, seed)
    na = nb = norb // 2
    S = Sector.molecular(norb, na, nb)
    hf = ((1 << na) - 1) | (((1 << nb) - 1) << norb)
    ans = ProductAnsatz.pair_doubles(norb, w.pair_double_ansatz(norb, count), S, hf)
    rows = seniority_rows(S, norb) if support else None

    def make(R):
        h, g = w.pes_point(h0, h1, g0, R)
        return EnergyGradient(PauliSum.jw_molecular(h, g, eps_drop=1e-12), S, ans, dtype=dtype, rows=rows)

    return S, ans, make, rows


def compare(prev, warm, min_train: int, target: float = TARGET):
    rows = []
    tot = {"previous": [0, 0, 0.0], "mlp": [0, 0, 0.0]}
    reached = {"previous": 0, "mlp": 0}
    for i, (a, b) in enumerate(zip(prev, warm)):
        e_ref = min(a.E, b.E)
        row = {"R": a.R, "E_ref": e_ref, "start": b.start,
               "start_error": {"previous": a.E_start - e_ref, "mlp": b.E_start - e_ref}}
        for name, r in (("previous", a), ("mlp", b)):
            hit = iterations_to(r, e_ref + target)
            row[name] = {"E": r.E, "nit": r.nit, "nfev": r.nfev, "seconds": r.seconds,
                         "to_target": None if hit is None else {"iterations": hit[0], "evaluations": hit[1],
                                                                  "seconds": hit[2]}}
            if i >= min_train:
                if hit is not None:
                    reached[name] += 1
                    tot[name][0] += hit[0]
                    tot[name][1] += hit[1]
                    tot[name][2] += hit[2]
        row["mlp"]["fit_seconds"] = b.fit_seconds
        row["mlp"]["E_guess"] = b.E_guess
        row["mlp"]["E_previous"] = b.E_previous
        rows.append(row)
    return rows, tot, reached


def run(norb: int = 8, npoints: int = 40, count: int = 200, dtype: str = "c128", seed: int | None = None,
        min_train: int = 3, fit_steps: int = 150, lr: float = 1e-3, maxiter: int = 300, ftol: float = 1e-10,
        window: int = 10, log=None, support: bool = False):
    import torch
    import workloads as w
    tdt = torch.complex128 if dtype == "c128" else torch.complex64
    seed = w.PES_SEED if seed is None else seed
    pts = [w.PES_POINTS[0] + (w.PES_POINTS[-1] - w.PES_POINTS[0]) * i / max(npoints - 1, 1) for i in range(npoints)]
    S, ans, make, supp = make_scan_problem(norb, count, tdt, seed, support)
    opt = dict(maxiter=maxiter, ftol=ftol, gtol=1e-7)
    t0 = time.perf_counter()
    prev = scan(make, pts, count, warm=None, opt=opt, log=log)
    t1 = time.perf_counter()
    ws = WarmStart(count, (pts[0], pts[-1]), hidden=256, max_points=max(npoints, 1), seed=seed, window=window)
    warm = scan(make, pts, count, warm=ws, min_train=min_train, fit_steps=fit_steps, lr=lr, opt=opt, log=log,
                reuse=prev[:min_train])
    t2 = time.perf_counter()
    rows, tot, reached = compare(prev, warm, min_train)
    n_eval = npoints - min_train
    fit_total = sum(r.fit_seconds for r in warm)
    return {
        "workload": f"pes-norb{norb}-({norb // 2}a,{norb // 2}b)-dim{S.dim}-K{count}",
        "evaluation": ("pauli_expect_rows on the C(norb, norb/2) = %d seniority-zero rows, rotations on the "
                       "full sector vector" % supp.numel()) if supp is not None else "pauli_expect on the full sector",
        "dtype": dtype, "points": npoints, "min_train": min_train, "window": window, "target_ha": TARGET,
        "points_compared": n_eval,
        "previous_start": {"iterations": tot["previous"][0], "evaluations": tot["previous"][1],
                           "seconds": tot["previous"][2], "reached": reached["previous"],
                           "scan_seconds": t1 - t0},
        "mlp_start": {"iterations": tot["mlp"][0], "evaluations": tot["mlp"][1], "seconds": tot["mlp"][2],
                      "reached": reached["mlp"], "scan_seconds": t2 - t1,
                      "fit_seconds": fit_total,
                      # the network's training counted against the learned arm
                      "seconds_with_fit": tot["mlp"][2] + fit_total,
                      "mlp_starts": sum(1 for r in warm if r.start == "mlp")},
        "rows": rows,
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--norb", type=int, default=8)
    ap.add_argument("--points", type=int, default=40)
    ap.add_argument("--count", type=int, default=200)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--min-train", type=int, default=3)
    ap.add_argument("--fit-steps", type=int, default=150,
                    help="Adam steps per refit (the network is refit from its previous weights after each point)")
    ap.add_argument("--maxiter", type=int, default=300)
    ap.add_argument("--window", type=int, default=10)
    ap.add_argument("--rows", action="store_true", help="include the per-point rows")
    ap.add_argument("--seniority-rows", action="store_true",
                    help="energies and gradients from the seniority-zero rows of H psi (pauli_expect_rows)")
    a = ap.parse_args(argv)
    out = run(a.norb, a.points, a.count, a.dtype, min_train=a.min_train, fit_steps=a.fit_steps, maxiter=a.maxiter,
              window=a.window, log=lambda m: print(m, file=sys.stderr, flush=True), support=a.seniority_rows)
    if not a.rows:
        out.pop("rows")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
