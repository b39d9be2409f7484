"""Persistent batched launch and the launch-shape autotuner: same results as the
single-state path (and the oracle), whatever shape is chosen."""
import math

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small_batch(ps):
    """Ragged batch: 2..7 orbitals, closed and open shell, one empty-ish sector."""
    specs = [(4, 2, 2, 1), (6, 3, 3, 2), (5, 2, 3, 3), (7, 3, 3, 4), (3, 1, 1, 5), (6, 2, 4, 6), (2, 1, 0, 7),
             (7, 4, 4, 8)]
    Hs, Ss, Ros, Sos, psis = [], [], [], [], []
    for norb, na, nb, seed in specs:
        h, g = w.molecular_integrals(norb, seed)
        Hs.append(ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12))
        Ros.append(oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12))
        Ss.append(ps.Sector.molecular(norb, na, nb))
        Sos.append(oracle.Sector.molecular(norb, na, nb))
        psis.append(w.random_state(Ss[-1].dim, 100 + seed))
    return Hs, Ss, Ros, Sos, psis


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_batch_matches_single_and_oracle(ps, small_batch, prec):
    import torch
    Hs, Ss, Ros, Sos, psis = small_batch
    dt = torch.complex128 if prec == "c128" else torch.complex64
    xs = [torch.from_numpy(p).to("cuda", dt) for p in psis]
    outs = [torch.empty_like(x) for x in xs]
    B = ps.Batch(Hs, Ss, dtype=dt)
    res = B.apply(xs, outs).cpu().numpy()
    tol = 1e-12 if prec == "c128" else 1e-5
    for b, (H, S, R, So, x) in enumerate(zip(Hs, Ss, Ros, Sos, xs)):
        xin = x.cpu().numpy().astype(np.complex128)
        ref = oracle.apply(So, R, xin)
        got = outs[b].cpu().numpy().astype(np.complex128)
        assert _rel(got, ref) <= tol, b
        E, n2 = oracle.expect(So, R, xin)
        assert abs(complex(res[b, 0], res[b, 1]) - E) <= (1e-12 if prec == "c128" else 1e-6)
        assert abs(res[b, 3] - np.vdot(xin, xin).real) <= 1e-12
    # expectation only (no output vectors) and determinism
    r2 = B.apply(xs).cpu().numpy()
    assert np.array_equal(r2, res)


def test_batch_tune_keeps_results(ps, small_batch):
    import torch
    Hs, Ss, Ros, Sos, psis = small_batch
    xs = [torch.from_numpy(p).to("cuda", torch.complex64) for p in psis]
    B = ps.Batch(Hs, Ss, dtype=torch.complex64)
    before = B.apply(xs).cpu().numpy()
    cfg = B.tune(xs, reps=2)
    assert cfg["cols_per_thread"] in (0, 1, 2, 4) and cfg["staged_rows"] in (0, 1, 2) and cfg["ms"] > 0
    after = B.apply(xs).cpu().numpy()
    assert np.allclose(after, before, rtol=1e-5, atol=1e-6)


def test_tune_single_and_cache(ps, tmp_path):
    import torch
    h, g = w.MOL12.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(6, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(6, 3, 3)
    So = oracle.Sector.molecular(6, 3, 3)
    cache = str(tmp_path / "tune.json")
    cfg = ps.tune(H, S, torch.complex64, reps=2, cache=cache)
    assert not cfg["cached"] and cfg["ms"] > 0
    # the cache is the C library's text file (pauli_tune_save)
    lines = [ln.split() for ln in open(cache).read().splitlines()]
    assert len(lines) == 1 and lines[0][0] == "paulisim-tune-v1" and lines[0][2] == "c64"
    assert int(lines[0][3]) == cfg["cols_per_thread"]
    assert ps.launch_config(H, S, torch.complex64)["cols_per_thread"] == cfg["cols_per_thread"]
    psi = w.random_state(S.dim, 3)
    x = torch.from_numpy(psi).to("cuda", torch.complex64)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    assert _rel(out, oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))) <= 1e-5
    # a fresh operator picks the cached shape without timing
    H2 = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    cfg2 = ps.tune(H2, S, torch.complex64, cache=cache)
    assert cfg2["cached"] and cfg2["cols_per_thread"] == cfg["cols_per_thread"]
    assert cfg2["row_split"] == cfg["row_split"]
    # an explicitly installed shape is used and still exact
    H3 = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    ps.prepare(H3, S)
    c = ps.LaunchConfig(cols_per_thread=1, staged_rows=2, row_split=3, direct=0, ranked=0, ms=0.0)
    ps._check(ps.lib().pauli_set_launch_config(H3._h, S._h, ps.C128, ps.C.byref(c)))
    got = ps.launch_config(H3, S, torch.complex128)
    assert (got["cols_per_thread"], got["staged_rows"], got["row_split"]) == (1, 2, 3)
    y = torch.from_numpy(psi).to("cuda", torch.complex128)
    assert _rel(ps.apply(H3, S, y).cpu().numpy(), oracle.apply(So, R, psi)) <= 1e-12
