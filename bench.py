"""Benchmark of the Pauli-sum operator-state hot path on one GB300 (replicas across GPUs).

Workload: the 24-qubit synthetic molecule (12 spatial orbitals, generator seed 0,
Jordan-Wigner, canonical reduction with eps_drop 1e-12: M = 29,737 terms in
G = 5,479 X-mask groups) applied to a seeded random unit state of the
(6 alpha, 6 beta) sector, D = 853,776.  One step = one pauli_apply (H psi)
with complex64 storage and FP32 group sums (the default) or complex128 / FP64.

metric: H|psi> term-amplitude updates per second, U / t, with
U = sum_k #{t in S : t XOR x_k in S} counted exactly from the canonical masks.

Prints one JSON line (see the end of main()).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

METRIC = "H|psi> term-amplitude updates/s"
UNIT = "updates/s"
L2_BYTES = 126 * 2 ** 20


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# workload bookkeeping (host side, not timed)
# ---------------------------------------------------------------------------
def count_updates(x: np.ndarray, n_lo: int, n_hi: int, k_lo: int, k_hi: int) -> int:
    """U = sum_k #{t in S : t ^ x_k in S} for a single product block (k_lo, k_hi):
    flipping the bits of a mask with m bits keeps the popcount of a string iff
    exactly m/2 of them are set, so a half contributes C(m, m/2) C(bits - m, k - m/2)."""
    def half_count(m, bits, k):
        if m % 2:
            return 0
        a = m // 2
        if k - a < 0 or k - a > bits - m:
            return 0
        return math.comb(m, a) * math.comb(bits - m, k - a)
    lomask = (1 << n_lo) - 1
    total = 0
    for xv in x.tolist():
        ml = bin(xv & lomask).count("1")
        mh = bin(xv >> n_lo).count("1")
        total += half_count(ml, n_lo, k_lo) * half_count(mh, n_hi, k_hi)
    return total


def measured_peaks():
    """(HBM GB/s, kind, max SM MHz) from MEASURED_PEAKS.json, else the fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured", d.get("sm_max_mhz", 2070.0)
    return 6800.0, "fallback", 2070.0


# Popcount results per SM per clock on sm_103a (CUDA throughput table; a probe on
# the GB300 measured 15.8).  One term-amplitude update of eq. reverse_sum needs one
# popcount parity, so SMs x 16 x clock is the update roof of the parity pipe.
POPC_PER_CLK_SM = 16


def profiled_traffic(name: str):
    """DRAM bytes per launch from the committed ncu capture, if the kernel sources
    still match the ones captured (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256()
    for s in d["sources"]:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return d["dram_bytes_per_launch"] if h.hexdigest() == d["sources_sha256"] else None


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over the ranks of the default process group (x itself
    without one): the job's step time is that of its slowest replica."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------
_ORACLE_CASE = {}


def headline_config(terms: int, groups: int, updates: int) -> dict:
    """The workload dict both arms print (the reference arm runs the same workload)."""
    return {"workload": "mol24: 24 qubits, 12 orbitals, seed 0, (6a,6b) sector D=853776",
            "terms": int(terms), "groups": int(groups), "updates_per_apply": int(updates),
            "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}


def _oracle_case():
    """The 24-qubit operator, sector and state on the oracle side (built once)."""
    if not _ORACLE_CASE:
        import oracle
        h, g = w.MOL24.integrals()
        R = oracle.jw_hamiltonian(12, h, g, eps_drop=1e-12)
        So = oracle.Sector.molecular(12, 6, 6)
        psi = w.random_state(So.dim, w.MOL24.psi_seed)
        _ORACLE_CASE.update(R=R, So=So, psi=psi, U=count_updates(R.x, 12, 12, 6, 6))
    return _ORACLE_CASE


def oracle_rate(seconds: float = 10.0, max_rows: int | None = None):
    """Oracle updates/s from the per-target definition on a bounded sample of rows."""
    import oracle
    case = _oracle_case()
    R, So, psi, U = case["R"], case["So"], case["psi"], case["U"]
    D = So.dim
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    oracle.apply_rows(So, R, psi, rng.integers(0, D, 64))
    per_row = (time.perf_counter() - t0) / 64
    nrows = max(64, int(seconds / per_row))
    if max_rows:
        nrows = min(nrows, max_rows)
    rows = rng.integers(0, D, nrows)
    t0 = time.perf_counter()
    oracle.apply_rows(So, R, psi, rows)
    dt = time.perf_counter() - t0
    est_apply_s = dt / nrows * D
    return U / est_apply_s, nrows, dt, est_apply_s


def run_reference(args, rank, world):
    if rank != 0:
        return
    vals = []
    # bounded: the whole run (warm-up + timed steps) takes about two minutes whatever
    # --steps / --warmup are; each step times a row sample of the same apply
    per_step = min(args.ref_seconds, max(0.05, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(seconds=min(1.0, per_step))
    t_all = time.perf_counter()
    info = None
    for _ in range(args.steps):
        v, nrows, dt, est = oracle_rate(seconds=per_step)
        vals.append(v)
        info = (nrows, dt, est)
    wall = time.perf_counter() - t_all
    value = statistics.median(vals)
    nrows, dt, est = info
    sample = (f"{nrows} random target rows of the 24-qubit (6a,6b) apply by the per-target definition "
              f"(sum_k C_k <t|P_k|psi>), {dt:.1f} s, scaled to one full apply ({est:.0f} s)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": headline_config(len(_oracle_case()["R"].x), len(np.unique(_oracle_case()["R"].x)),
                                  _oracle_case()["U"]),
        "note": "the oracle on host cores; the config's l2 entry describes the GPU arm's timing",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2606_28952_gb300 as ps

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    tdt = torch.complex64 if args.dtype == "c64" else torch.complex128
    esize = 8 if args.dtype == "c64" else 16
    h, g = w.MOL24.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(12, 6, 6)
    ps.prepare(H, S)
    install_launch(ps, H, S, tdt, args.launch)
    x_can, _, _ = H.export()
    U = count_updates(x_can, 12, 12, 6, 6)
    # group-level count U_g = sum_g #{t in S : t ^ x_g in S}: one source amplitude read per
    # (target, group) pair that has a contribution
    U_g = count_updates(np.unique(np.asarray(x_can, dtype=np.uint64)), 12, 12, 6, 6)
    psi_np = w.random_state(S.dim, w.MOL24.psi_seed)
    psi = torch.from_numpy(psi_np).to(dev, tdt)
    out = torch.empty_like(psi)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ps.apply(H, S, psi, out)
    torch.cuda.synchronize()

    # device-timed region: inputs resident, L2 flushed between timed steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        ps.apply(H, S, psi, out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    time.sleep(0.2)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    times_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_step = max_over_ranks(sum(times_ms) / len(times_ms) / 1e3, dist, dev)
    value = world * U / t_step

    # end to end: pinned host psi -> device -> apply -> host, every step
    host_in = torch.from_numpy(psi_np).to(tdt).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dev_in = torch.empty_like(psi)
    for _ in range(max(3, args.warmup)):
        dev_in.copy_(host_in, non_blocking=True)
        ps.apply(H, S, dev_in, out)
        host_out.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(10, args.steps // 4)
    e0.record(stream)
    for _ in range(e2e_steps):
        dev_in.copy_(host_in, non_blocking=True)
        ps.apply(H, S, dev_in, out)
        host_out.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3 / e2e_steps
    bytes_io = S.dim * esize

    # roofline bookkeeping for the apply kernel
    hbm_peak, peak_kind, sm_mhz_max = measured_peaks()
    table_bytes = H.m * (8 + 8 + 2 * (4 if args.dtype == "c64" else 8)) + H.n_groups * 16
    alg_bytes = 2 * S.dim * esize + table_bytes
    achieved_gbs = alg_bytes / t_step / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    popc_peak = sms * POPC_PER_CLK_SM * sm_mhz_max * 1e6 / 1e9  # G parities / s
    achieved_gups = U / t_step / 1e9

    # side measurements (not the headline): expectation value and the other precision
    res = torch.empty(4, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ps.expect(H, S, psi, result=res)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(10):
        ps.expect(H, S, psi, result=res)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_expect = ev0.elapsed_time(ev1) / 1e3 / 10
    other = torch.complex128 if tdt == torch.complex64 else torch.complex64
    psi_o = psi.to(other)
    out_o = torch.empty_like(psi_o)
    ps.apply(H, S, psi_o, out_o)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(5):
        ps.apply(H, S, psi_o, out_o)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_other = ev0.elapsed_time(ev1) / 1e3 / 5

    # kernels per pauli_apply: the gather, plus the fixed-order sum of the row-piece split
    lc = ps.launch_config(H, S, tdt)
    launches_per_apply = 2 if lc["row_split"] > 1 and not lc["direct"] else 1

    # side measurement: one pair-double rotation on the 32-qubit (8a,8b) sector
    # (165,636,900 amplitudes, 1.3 GB complex64) against the HBM roof of the
    # amplitudes it touches (read + write of every pair with f != 0)
    rot = None
    if not args.no_rotate:
        norb = w.PES_NORB
        Sr = ps.Sector.molecular(norb, norb // 2, norb // 2)
        Gr = ps.PauliSum.jw_fermion(2 * norb, w.pair_double_generator(norb, 0, norb - 1))
        phi = torch.zeros(Sr.dim, dtype=torch.complex64, device=dev)
        phi.fill_(1.0 / math.sqrt(Sr.dim))
        ps.rotate(Gr, Sr, 0.1, phi)
        torch.cuda.synchronize()
        nrot = 20
        ev0.record(stream)
        for _ in range(nrot):
            ps.rotate(Gr, Sr, 0.1, phi)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_rot = ev0.elapsed_time(ev1) / 1e3 / nrot
        # pairs with f != 0: orbital 0 doubly occupied and orbital norb-1 empty, or the
        # reverse; the other norb-2 orbitals hold (k-1) alpha and (k-1) beta electrons
        k = norb // 2
        touched = 2 * math.comb(norb - 2, k - 1) ** 2
        rot_bytes = 2 * 8 * touched
        rot = {"ms": t_rot * 1e3, "sector_dim": Sr.dim, "touched_amplitudes": touched,
               "compulsory_bytes": rot_bytes, "achieved_gbs": rot_bytes / t_rot / 1e9,
               "hbm_frac": rot_bytes / t_rot / 1e9 / hbm_peak}
        del phi
        torch.cuda.empty_cache()

    # side measurements on the other workloads (same build, same run): the
    # bandwidth-graded lattice applies, the persistent batch against sequential
    # launches in both precisions, and the 32-qubit molecule
    side_wl = {}
    if not args.no_side:
        side_wl["xxz30_full_apply_c64"] = xxz_apply_measure(ps, dev, w.XXZ_SITES, False, reps=10)
        side_wl["xxz30_sz0_apply_c64"] = xxz_apply_measure(ps, dev, w.XXZ_SITES, True, reps=20)
        side_wl["batched64_c64"] = batched_measure(
            ps, dev, warmup=1, steps=3, seeded_states=False,
            shape=ps.LaunchConfig(cols_per_thread=4, staged_rows=1, row_split=1, direct=0, ranked=1, ms=0.0),
            alt_shapes={"per_state_shape_groups": ps.LaunchConfig(cols_per_thread=0, staged_rows=1, row_split=1,
                                                                  direct=0, ranked=0, ms=0.0)})
        side_wl["mol32_apply_c64"] = mol32_apply_measure(ps, dev, reps=2)
        side_wl["uccsd_trotter_24q_c64"] = uccsd_measure(ps, dev, reps=5)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, nrows, dt, est = oracle_rate(seconds=args.ref_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nrows} random target rows by the per-target definition, {dt:.1f} s, "
                         f"scaled to one full apply ({est:.0f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64/f32" if args.dtype == "c64" else "c128/f64",
            "data": "synthetic",
            "config": headline_config(H.m, H.n_groups, U),
            "roofline": {"bound": "alu", "achieved": achieved_gups, "peak": popc_peak, "unit": "Gupd/s",
                         "frac": achieved_gups / popc_peak,
                         "eff_hbm": achieved_gbs / hbm_peak, "eff_hbm_achieved_gbs": achieved_gbs,
                         "gather_gbs": U_g * esize / t_step / 1e9, "gather_pairs_per_apply": U_g,
                         "eff_hbm_compulsory_bytes": alg_bytes, "eff_hbm_peak_gbs": hbm_peak,
                         "traffic": profiled_traffic("k_apply_mol24_c64.json") if args.dtype == "c64" else None,
                         "note": (f"updates U={U} per launch / CUDA-event step time (the step is the gather "
                                  f"kernel plus, when rows are split, its fixed-order combine: "
                                  f"{launches_per_apply} launch(es) per step); peak = {sms} SMs x "
                                  f"{POPC_PER_CLK_SM} popcounts/clk x {sm_mhz_max:.0f} MHz (one parity per "
                                  f"update); HBM view: {alg_bytes} compulsory bytes -> {achieved_gbs:.2f} GB/s "
                                  f"= {achieved_gbs / hbm_peak:.5f} of {peak_kind} {hbm_peak} GB/s")},
            "cpu_baseline": cpu,
            "e2e": {"value": world * U / t_e2e, "unit": UNIT, "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io},
            "gpu_launches": args.steps * launches_per_apply,
            "clocks": clk,
            "side": {"expect_ms": t_expect * 1e3, f"apply_{'c128' if tdt == torch.complex64 else 'c64'}_ms": t_other * 1e3,
                     "step_times_ms_min_max": [min(times_ms), max(times_ms)],
                     "launch_shape": lc, "rotate_pair_double_32q_c64": rot,
                     "fp32_vs_fp64_24q": {"c64_ms": t_step * 1e3 if tdt == torch.complex64 else t_other * 1e3,
                                          "c128_ms": t_other * 1e3 if tdt == torch.complex64 else t_step * 1e3},
                     **side_wl},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def install_launch(ps, H, S, tdt, spec: str):
    """--launch cols_per_thread,staged_rows,row_split,direct,ranked: install that
    shape (pauli_set_launch_config) instead of the heuristic one."""
    if not spec:
        return
    t, nb, sp, d, r = (int(v) for v in spec.split(","))
    ps.set_launch_config(H, S, tdt, ps.LaunchConfig(cols_per_thread=t, staged_rows=nb, row_split=sp, direct=d,
                                                    ranked=r, ms=0.0))


def run_xxz(args, rank, world, local_rank):
    """30-site open XXZ chain (seed 1), Neel start: one H|psi> timing and Krylov
    real-time steps (m = 20, dt = 0.05, the step replayed as a CUDA graph), in the
    full 2^30 space (complex64, 8.6 GB per vector) or the Sz = 0 block sector."""
    import torch
    import paper_2606_28952_gb300 as ps

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = args.sites or w.XXZ_SITES
    x, z, cre, cim = w.xxz_terms(n, w.XXZ_SEED)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim)
    if args.workload == "xxz30":
        S = ps.Sector.full(n, args.n_lo or 10)
        label = f"xxz{n} full space 2^{n}, split {S.n_lo if S.n_lo else 10}|{n - (args.n_lo or 10)}"
    else:
        nl = args.n_lo or 15  # 15|15: 16 blocks (k, 15-k); fastest split measured for this chain
        S = ps.Sector(n, ps.BLOCKS, nl, [(k, n // 2 - k) for k in range(0, min(nl, n // 2) + 1) if n // 2 - k <= n - nl])
        label = f"xxz{n} Sz=0 blocks, split {nl}|{n - nl}, D={S.dim}"
    ps.prepare(H, S)
    install_launch(ps, H, S, torch.complex64, args.launch)
    xc, _, _ = H.export()
    # term updates of one apply in the full space = M * 2^n; in a sector count per term
    if S.kind == ps.FULL:
        U = H.m * S.dim
    else:
        U = None
    stream = torch.cuda.current_stream()
    # --- one apply: psi (random) -> H psi, inputs far larger than L2 ---
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    psi = torch.randn(S.dim, dtype=torch.complex64, device=dev, generator=g)
    out = torch.empty_like(psi)
    for _ in range(args.warmup):
        ps.apply(H, S, psi, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    napp = max(3, args.steps)
    e0.record(stream)
    for _ in range(napp):
        ps.apply(H, S, psi, out)
    e1.record(stream)
    torch.cuda.synchronize()
    t_apply = e0.elapsed_time(e1) / 1e3 / napp
    del out
    hbm_peak, peak_kind, _ = measured_peaks()
    apply_bytes = 2 * S.dim * 8 + H.m * 24 + H.n_groups * 16
    if args.krylov_steps == 0:
        # apply only (e.g. for a profiler capture of the gather at a reduced size)
        if rank == 0:
            print(json.dumps({
                "metric": "H|psi> term-amplitude updates/s" if U else "H|psi> applies/s",
                "value": (U / t_apply) if U else 1.0 / t_apply, "unit": "updates/s" if U else "applies/s",
                "n_gpus": world, "steps": napp, "ms_per_step": t_apply * 1e3, "dtype": "c64/f32",
                "data": "synthetic", "config": {"workload": label, "terms": H.m, "groups": H.n_groups},
                "apply": {"ms": t_apply * 1e3, "compulsory_bytes": apply_bytes,
                          "hbm_frac": apply_bytes / t_apply / 1e9 / hbm_peak,
                          "peak": f"{peak_kind} {hbm_peak} GB/s"}}), flush=True)
        return
    # --- Krylov steps from the Neel state ---
    psi.zero_()
    neel = torch.tensor([w.neel_config(n)], dtype=torch.int64, device=dev)
    psi[S.rank(neel)[0].item()] = 1.0
    e_start = ps.expect(H, S, psi)[0].item()
    k = ps.Krylov(H, S, m=20, dtype=torch.complex64)
    k.step(psi, 0.05, nsteps=1, graph=True)  # capture
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    e0.record(stream)
    k.step(psi, 0.05, nsteps=args.krylov_steps, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = e0.elapsed_time(e1) / 1e3 / args.krylov_steps
    nrm = torch.linalg.vector_norm(psi).item()
    e_end = ps.expect(H, S, psi)[0].item()
    step_vectors = 9 * 20 + 4
    line = {
        "metric": "Krylov real-time steps/s (m=20, dt=0.05)", "value": 1.0 / t_step, "unit": "steps/s",
        "n_gpus": world, "steps": args.krylov_steps, "ms_per_step": t_step * 1e3, "dtype": "c64/f32, f64 scalars",
        "data": "synthetic", "config": {"workload": label, "terms": H.m, "groups": H.n_groups},
        "apply": {"ms": t_apply * 1e3, "updates_per_s": (U / t_apply) if U else None,
                  "compulsory_bytes": apply_bytes, "achieved_gbs": apply_bytes / t_apply / 1e9,
                  "hbm_frac": apply_bytes / t_apply / 1e9 / hbm_peak, "peak": f"{peak_kind} {hbm_peak} GB/s"},
        "step_bytes_compulsory": step_vectors * S.dim * 8,
        "step_hbm_frac": step_vectors * S.dim * 8 / t_step / 1e9 / hbm_peak,
        "norm_after": nrm, "energy_start": e_start, "energy_after": e_end,
        "steps_total": 1 + args.krylov_steps, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_measure(ps, dev, warmup: int, steps: int, tune_reps: int = 2, shape=None, seeded_states=True,
                    alt_shapes=None):
    """64 independent synthetic molecules (n_orb ~ U{8..14}, half filling): one
    persistent complex64 launch of H_b psi_b + <H>_b (FP64 reductions) against 64
    sequential complex128 and 64 sequential complex64 pauli_expect calls, all on
    this build.  The launch shape comes from the autotuner (tune_reps > 0) or is
    installed (shape = LaunchConfig)."""
    import torch
    mols = w.batched_states(64, 3)
    t0 = time.perf_counter()
    Hs, Ss, U, Bc = [], [], 0, 0
    for m in mols:
        h, g = m.integrals()
        H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
        S = ps.Sector.molecular(m.norb, m.n_alpha, m.n_beta)
        Hs.append(H)
        Ss.append(S)
        xc, _, _ = H.export()
        U += count_updates(xc, m.norb, m.norb, m.n_alpha, m.n_beta)
        Bc += 2 * S.dim * 8 + H.m * 24 + H.n_groups * 16
    t_build = time.perf_counter() - t0
    dims = [S.dim for S in Ss]
    if seeded_states:
        psis = [torch.from_numpy(w.random_state(S.dim, m.psi_seed)).to(dev) for S, m in zip(Ss, mols)]  # c128
    else:
        gen = torch.Generator(device=dev)
        gen.manual_seed(2000)
        psis = []
        for S in Ss:
            v = torch.randn(S.dim, dtype=torch.complex128, device=dev, generator=gen)
            psis.append(v / torch.linalg.vector_norm(v))
    x64 = [p.to(torch.complex64) for p in psis]
    outs = [torch.empty_like(x) for x in x64]
    B = ps.Batch(Hs, Ss, dtype=torch.complex64)
    if shape is not None:
        B.set_launch_config(shape)
        cfg = dict(B.launch_config(), source="installed")
    else:
        cfg = dict(B.tune(x64, outs, reps=tune_reps), source="autotuner")
    stream = torch.cuda.current_stream()
    res = torch.empty((64, 4), dtype=torch.float64, device=dev)
    for _ in range(warmup):
        B.apply(x64, outs, res)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(steps):
        B.apply(x64, outs, res)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_batch = e0.elapsed_time(e1) / 1e3 / steps
    # other installed shapes, same states (informational)
    alt = {}
    for name, c in (alt_shapes or {}).items():
        B.set_launch_config(c)
        B.apply(x64, outs, res)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            B.apply(x64, outs, res)
        e1.record(stream)
        torch.cuda.synchronize()
        alt[name] = {"ms": e0.elapsed_time(e1) / steps, "launches": int(B.launch_config()["ms"])}
    # 64 sequential FP64 launches (one pauli_expect with H psi per state)
    r128 = torch.empty((64, 4), dtype=torch.float64, device=dev)
    h128 = [torch.empty_like(p) for p in psis]
    for b in range(64):
        ps.expect(Hs[b], Ss[b], psis[b], hpsi_out=h128[b], result=r128[b])
    torch.cuda.synchronize()
    e0.record(stream)
    for b in range(64):
        ps.expect(Hs[b], Ss[b], psis[b], hpsi_out=h128[b], result=r128[b])
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    del h128
    # and 64 sequential complex64 launches with each state's default launch shape
    r64 = torch.empty((64, 4), dtype=torch.float64, device=dev)
    for b in range(64):
        ps.expect(Hs[b], Ss[b], x64[b], hpsi_out=outs[b], result=r64[b])
    torch.cuda.synchronize()
    e0.record(stream)
    for b in range(64):
        ps.expect(Hs[b], Ss[b], x64[b], hpsi_out=outs[b], result=r64[b])
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq64 = e0.elapsed_time(e1) / 1e3
    dE = (res[:, 0] - r128[:, 0]).abs().max().item()
    hbm_peak, peak_kind, sm_mhz_max = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    popc_peak = sms * POPC_PER_CLK_SM * sm_mhz_max * 1e6
    return {
        "ms": t_batch * 1e3, "updates_per_s": U / t_batch, "popc_roof_frac": U / t_batch / popc_peak,
        "compulsory_bytes": Bc, "hbm_frac": Bc / t_batch / 1e9 / hbm_peak,
        "sum_dim": int(sum(dims)), "max_dim": int(max(dims)), "min_dim": int(min(dims)),
        "updates_per_batch": U, "shape": cfg, "build_s": t_build, "steps": steps,
        "sequential_c128_ms": t_seq * 1e3, "speedup_vs_sequential_c128": t_seq / t_batch,
        "sequential_c64_ms": t_seq64 * 1e3, "speedup_vs_sequential_c64": t_seq64 / t_batch,
        "max_energy_diff_c64_vs_c128_Ha": dE, "clocks": clk, "peak": f"{peak_kind} {hbm_peak} GB/s",
        "other_shapes": alt or None,
    }


def run_batched(args, rank, world, local_rank):
    """The batched workload on its own (autotuned shape, seeded states)."""
    import torch
    import paper_2606_28952_gb300 as ps

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    r = batched_measure(ps, dev, args.warmup, args.steps)
    line = {
        "metric": METRIC, "value": r["updates_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "ms_per_step": r["ms"], "dtype": "c64/f32, f64 reductions", "data": "synthetic",
        "config": {"workload": "64 molecules, n_orb ~ U{8..14} (seed 3), half filling, H psi + <H> per state",
                   "sum_dim": r["sum_dim"], "max_dim": r["max_dim"], "min_dim": r["min_dim"],
                   "updates_per_batch": r["updates_per_batch"], "tuned_shape": r["shape"], "build_s": r["build_s"]},
        **{k: r[k] for k in ("sequential_c128_ms", "speedup_vs_sequential_c128", "sequential_c64_ms",
                             "speedup_vs_sequential_c64", "max_energy_diff_c64_vs_c128_Ha", "clocks", "hbm_frac",
                             "popc_roof_frac")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def xxz_apply_measure(ps, dev, n: int, sz0: bool, n_lo: int = 0, warmup: int = 3, reps: int = 10,
                      launch: str = ""):
    """One H psi of the open XXZ chain (seed 1) on a random complex64 state, in the
    full 2^n space or the Sz = 0 block sector; CUDA events, clocks sampled.
    Inputs are far larger than L2 at 30 sites (8.6 GB / 1.24 GB per vector)."""
    import torch
    x, z, cre, cim = w.xxz_terms(n, w.XXZ_SEED)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim)
    if not sz0:
        S = ps.Sector.full(n, n_lo or 10)
        label = f"xxz{n} full space 2^{n}"
    else:
        nl = n_lo or n // 2
        S = ps.Sector(n, ps.BLOCKS, nl, [(k, n // 2 - k) for k in range(0, min(nl, n // 2) + 1) if n // 2 - k <= n - nl])
        label = f"xxz{n} Sz=0 blocks, split {nl}|{n - nl}, D={S.dim}"
    ps.prepare(H, S)
    install_launch(ps, H, S, torch.complex64, launch)
    U = H.m * S.dim if S.kind == ps.FULL else None
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    psi = torch.randn(S.dim, dtype=torch.complex64, device=dev, generator=gen)
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ps.apply(H, S, psi, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.2)
    e0.record(stream)
    for _ in range(reps):
        ps.apply(H, S, psi, out)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_apply = e0.elapsed_time(e1) / 1e3 / reps
    hbm_peak, peak_kind, _ = measured_peaks()
    apply_bytes = 2 * S.dim * 8 + H.m * 24 + H.n_groups * 16
    r = {"workload": label, "dim": S.dim, "terms": H.m, "groups": H.n_groups, "ms": t_apply * 1e3, "reps": reps,
         "updates_per_s": (U / t_apply) if U else None, "compulsory_bytes": apply_bytes,
         "achieved_gbs": apply_bytes / t_apply / 1e9, "hbm_frac": apply_bytes / t_apply / 1e9 / hbm_peak,
         "peak": f"{peak_kind} {hbm_peak} GB/s", "launch_shape": ps.launch_config(H, S), "clocks": clk}
    del psi, out
    torch.cuda.empty_cache()
    return r


def uccsd_measure(ps, dev, reps: int = 5):
    """The 24-qubit molecule's UCCSD generators (1,818 single and double
    excitations): one Trotter step psi <- prod_k exp(-i theta_k G_k) psi applied
    tile by tile (pauli_rotseq) against 1,818 separate rotations
    (pauli_rotate_seq), complex64, random angles in [-0.3, 0.3]; and the ADAPT
    pool gradients of all 1,818 generators at a random state (one launch)."""
    import torch
    norb, na, nb = 12, 6, 6
    pool = w.uccsd_trotter_order(w.uccsd_pool(norb, na, nb), norb)
    gens = [ps.PauliSum.jw_fermion(2 * norb, t) for _, t in pool]
    S = ps.Sector.molecular(norb, na, nb)
    h, g = w.MOL24.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    thetas = np.random.default_rng(24).uniform(-0.3, 0.3, len(gens))
    Q = ps.RotSeq(gens, S)
    psi = torch.from_numpy(w.random_state(S.dim, 24)).to(dev, torch.complex64)
    x = psi.clone()
    stream = torch.cuda.current_stream()
    Q.apply(thetas, x)
    ps.rotate_seq(gens, S, thetas, x)  # first use builds the pair tables
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        Q.apply(thetas, x)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fused = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for _ in range(reps):
        ps.rotate_seq(gens, S, thetas, x)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / reps
    P = ps.Pool(gens, S)
    hx = torch.empty_like(psi)
    ps.expect(H, S, psi, hpsi_out=hx)
    out = torch.empty(len(gens), dtype=torch.float64, device=dev)
    P.gradients(psi, hx, out)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        P.gradients(psi, hx, out)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pool = e0.elapsed_time(e1) / reps
    info = Q.info(torch.complex64)
    return {"generators": len(gens), "fused_launches": info["launches"], "fused_ms": t_fused,
            "separate_rotations_ms": t_seq, "speedup": t_seq / t_fused, "pool_gradients_ms": t_pool,
            "pool_gradients_per_s": len(gens) / t_pool * 1e3}


def mol32_apply_measure(ps, dev, reps: int = 2):
    """One H psi of the 32-qubit PES molecule (16 orbitals, (8a,8b), D = 165,636,900,
    complex64, default launch shape) at the scan's R = 1.14 point."""
    import torch
    norb = w.PES_NORB
    h0, h1, g0 = w.pes_integrals(norb, w.PES_SEED)
    h, g = w.pes_point(h0, h1, g0, w.PES_POINTS[10])
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, norb // 2, norb // 2)
    ps.prepare(H, S)
    xc, _, _ = H.export()
    U = count_updates(xc, norb, norb, norb // 2, norb // 2)
    gen = torch.Generator(device=dev)
    gen.manual_seed(32)
    psi = torch.randn(S.dim, dtype=torch.complex64, device=dev, generator=gen)
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    ps.apply(H, S, psi, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(reps):
        ps.apply(H, S, psi, out)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3 / reps
    _, _, sm_mhz_max = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    r = {"workload": "32-qubit PES molecule, 16 orbitals, (8a,8b), D=165636900, R=1.14", "terms": H.m,
         "groups": H.n_groups, "updates_per_apply": U, "ms": t * 1e3, "updates_per_s": U / t,
         "popc_roof_frac": U / t / (sms * POPC_PER_CLK_SM * sm_mhz_max * 1e6),
         "launch_shape": ps.launch_config(H, S), "clocks": clk}
    del psi, out
    torch.cuda.empty_cache()
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["mol24", "xxz30", "xxz30-sz0", "batched64"], default="mol24")
    ap.add_argument("--n-lo", type=int, default=0)
    ap.add_argument("--sites", type=int, default=0, help="XXZ chain length (default 30; smaller for profiling)")
    ap.add_argument("--krylov-steps", type=int, default=5)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c64")
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rotate", action="store_true", help="skip the 32-qubit rotation side measurement")
    ap.add_argument("--no-side", action="store_true", help="skip the other workloads' side measurements")
    ap.add_argument("--launch", default="", help="cols_per_thread,staged_rows,row_split,direct,ranked of the apply")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched64":
        run_batched(args, rank, world, local_rank)
    elif args.workload != "mol24":
        run_xxz(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
