"""Oracle parity of the launch shapes and sizes that the benchmarks run.

* every launch shape the launch-shape interface can install on a mid-size
  single-block sector (10 orbitals, (5a,5b), D = 63,504): columns per thread,
  pattern- vs rank-staged rows, staged rows in flight, row splits, the list
  gather, and the direct gather on a small lattice operator; the shape that
  actually ran is read back and checked;
* the direct gather on a fixed-N sector of several blocks, with an operator
  whose strings keep a row in its block, move it to another block, or leave
  the sector;
* the 32-qubit (8a,8b) sector (D = 165,636,900) with its default shape (rows
  staged by rank, 8 columns per thread) on sampled target rows;
* the 64-molecule persistent batch at full size (8-14 orbitals) with the
  autotuned shape and both staging layouts, sampled rows of every state;
* the 24-qubit molecule on a 5% row sample plus the first and last target of
  every 16th row.

Element-by-element against the oracle on the same (dtype-rounded) inputs:
relative error of the sampled H psi entries <= 1e-12 (complex128) and 1e-5
(complex64).  The oracle's per-target definition runs in host threads (its C
calls release the interpreter lock)."""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _tdt(name):
    import torch
    return torch.complex128 if name == "c128" else torch.complex64


def _rounded(psi, dt):
    """The input as the device sees it (complex64 rounding), back in complex128."""
    return psi if dt == "c128" else psi.astype(np.complex64).astype(np.complex128)


def oracle_rows(So, R, psi, rows, nthreads=None):
    """oracle.apply_rows over row chunks in host threads."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    nthreads = nthreads or min(32, os.cpu_count() or 4)
    chunks = [c for c in np.array_split(rows, max(1, min(len(rows), 4 * nthreads))) if len(c)]
    with cf.ThreadPoolExecutor(nthreads) as ex:
        parts = list(ex.map(lambda c: oracle.apply_rows(So, R, psi, c), chunks))
    return np.concatenate(parts) if parts else np.zeros(0, np.complex128)


def _gather(t, rows):
    import torch
    idx = torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int64)).to(t.device)
    return t.index_select(0, idx).cpu().numpy().astype(np.complex128)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------------------
# launch-shape sweep, 10 orbitals (5a,5b)
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def mol20():
    norb, na, nb = 10, 5, 5
    h, g = w.molecular_integrals(norb, 4)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    So = oracle.Sector.molecular(norb, na, nb)
    psi = w.random_state(So.dim, 41)
    refs = {dt: (_rounded(psi, dt), oracle_rows(So, R, _rounded(psi, dt), np.arange(So.dim))) for dt in TOL}
    E = {dt: oracle.expect(So, R, refs[dt][0])[0] for dt in TOL}
    return h, g, R, So, psi, refs, E


def _expected_shape(tpt, nbuf, split, ranked):
    """The shape apply_config realises for a staged request: 8 columns per
    thread exist only for rank-staged rows and one staged row."""
    if tpt == 8 and not ranked:
        tpt = 4
    if tpt == 8:
        nbuf = 1
    return tpt, nbuf, ranked


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_launch_shape_sweep_10_orbitals(ps, mol20, dt):
    import torch
    h, g, R, So, psi, refs, E = mol20
    xin, ref = refs[dt]
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(10, 5, 5)
    ps.prepare(H, S)
    x = torch.from_numpy(xin).to("cuda", _tdt(dt))
    etol = 1e-12 if dt == "c128" else 1e-6
    seen = set()
    shapes = [(t, nb, sp, 0, rk) for t in (1, 2, 4, 8) for rk in (0, 1) for nb in (1, 2) for sp in (1, 4, 16)]
    shapes += [(1, 1, sp, 3, 0) for sp in (1, 4, 16)]
    for tpt, nbuf, split, direct, ranked in shapes:
        c = ps.LaunchConfig(cols_per_thread=tpt, staged_rows=nbuf, row_split=split, direct=direct, ranked=ranked,
                            ms=0.0)
        ps.set_launch_config(H, S, _tdt(dt), c)
        got = ps.launch_config(H, S, _tdt(dt))
        if direct == 3:
            assert got["direct"] == 3 and 1 <= got["row_split"] <= split, got
        else:
            et, en, er = _expected_shape(tpt, nbuf, split, ranked)
            assert (got["cols_per_thread"], got["staged_rows"], got["ranked"], got["direct"]) == (et, en, er, 0), \
                (tpt, nbuf, split, ranked, got)
            assert 1 <= got["row_split"] <= split
        key = tuple(got[k] for k in ("cols_per_thread", "staged_rows", "row_split", "direct", "ranked"))
        seen.add(key)
        out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
        assert _rel(out, ref) <= TOL[dt], (key, _rel(out, ref))
        r = ps.expect(H, S, x).cpu().numpy()
        assert abs(complex(r[0], r[1]) - E[dt]) <= etol, key
    # the 8-column rank-staged kernel (the one the 32-qubit sector runs) was among them
    assert any(k[0] == 8 and k[4] == 1 for k in seen)
    assert len(seen) >= 20


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["full16", "sz0_16"])
def test_direct_gather_shapes(ps, dt, kind):
    """The direct gather (small operators) with every columns-per-thread value,
    and the staged gather on the same operator."""
    import torch
    n = 16
    x, z, cre, cim = w.xxz_terms(n, 1)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim)
    R = oracle.build_sum(n, x, z, None, cre, cim)
    if kind == "full16":
        S = ps.Sector.full(n, 8)
        So = oracle.Sector.full(n)
    else:
        blocks = [(k, 8 - k) for k in range(9)]
        S = ps.Sector(n, ps.BLOCKS, 8, blocks)
        So = oracle.Sector(n, oracle.BLOCKS, 8, blocks)
    psi = _rounded(w.random_state(S.dim, 17), dt)
    ref = oracle.apply(So, R, psi)
    Eref = oracle.expect(So, R, psi)[0]
    ps.prepare(H, S)
    xt = torch.from_numpy(psi).to("cuda", _tdt(dt))
    for tpt in (1, 2, 4, 8):
        for direct in (1, 0):
            c = ps.LaunchConfig(cols_per_thread=tpt, staged_rows=1, row_split=1, direct=direct, ranked=0, ms=0.0)
            ps.set_launch_config(H, S, _tdt(dt), c)
            got = ps.launch_config(H, S, _tdt(dt))
            assert got["direct"] == direct and got["cols_per_thread"] == min(tpt, 4), got
            out = ps.apply(H, S, xt).cpu().numpy().astype(np.complex128)
            assert _rel(out, ref) <= TOL[dt], (tpt, direct)
            r = ps.expect(H, S, xt).cpu().numpy()
            assert abs(complex(r[0], r[1]) - Eref) <= (1e-12 if dt == "c128" else 1e-5) * max(1.0, abs(Eref))


def _block_changing_terms(n, n_lo, seed, real):
    """XZ-form strings whose X masks lie in the high half only (one bit: the row
    moves to a block of another low-half class, where no column of the target's
    row has a source; two bits: it stays in its class and the source column is the
    target's own), in the low half only, or in both, with random Z masks, plus
    diagonal strings."""
    rng = np.random.default_rng(seed)
    hi_bits = np.arange(n_lo, n)
    xs, zs, cre, cim = [], [], [], []

    def add(xm, k):
        for _ in range(k):
            xs.append(xm)
            zs.append(int(rng.integers(0, 1 << n)))
            cre.append(rng.normal())
            cim.append(0.0 if real else rng.normal())

    add(0, 6)
    for _ in range(6):
        add(1 << int(rng.choice(hi_bits)), 2)
    for _ in range(6):
        a, b = rng.choice(hi_bits, 2, replace=False)
        add((1 << int(a)) | (1 << int(b)), 2)
    for _ in range(6):
        add(int(rng.integers(1, 1 << n_lo)), 2)
    for _ in range(6):
        add(int(rng.integers(1, 1 << n_lo)) | (1 << int(rng.choice(hi_bits))), 2)
    return np.array(xs, np.uint64), np.array(zs, np.uint64), np.array(cre), np.array(cim)


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("real", [True, False])
def test_direct_gather_block_changes(ps, dt, real):
    """The direct gather on a fixed-N sector of several blocks (20 qubits, N = 10,
    12 low bits: rows of up to 924 columns, several column tiles at one column a
    thread), every columns-per-thread value, against the oracle and the staged gather."""
    import torch
    n, n_lo, N = 20, 12, 10
    x_, z_, cre, cim = _block_changing_terms(n, n_lo, 31 + int(real), real)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim, form=ps.XZ)
    R = oracle.build_sum(n, x_, z_, None, cre, cim, letter_form=False)
    blocks = [(k, N - k) for k in range(N + 1) if k <= n_lo and N - k <= n - n_lo]
    S = ps.Sector(n, ps.BLOCKS, n_lo, blocks)
    So = oracle.Sector(n, oracle.BLOCKS, n_lo, blocks)
    assert S.dim == So.dim == math.comb(n, N)
    psi = _rounded(w.random_state(S.dim, 23), dt)
    ref = oracle.apply(So, R, psi)
    E = complex(np.vdot(psi, ref))
    ps.prepare(H, S)
    xt = torch.from_numpy(psi).to("cuda", _tdt(dt))
    for tpt in (1, 2, 4):
        for direct in (1, 0):
            c = ps.LaunchConfig(cols_per_thread=tpt, staged_rows=1, row_split=1, direct=direct, ranked=0, ms=0.0)
            ps.set_launch_config(H, S, _tdt(dt), c)
            got = ps.launch_config(H, S, _tdt(dt))
            assert got["direct"] == direct and got["cols_per_thread"] == tpt, got
            out = ps.apply(H, S, xt).cpu().numpy().astype(np.complex128)
            assert _rel(out, ref) <= TOL[dt], (tpt, direct)
            r = ps.expect(H, S, xt).cpu().numpy()
            assert abs(complex(r[0], r[1]) - E) <= (1e-12 if dt == "c128" else 1e-5) * max(1.0, abs(E)), (tpt, direct)


# ----------------------------------------------------------------------------
# 32 qubits, (8a,8b): the default shape on sampled rows
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def mol32():
    norb = w.PES_NORB
    h0, h1, g0 = w.pes_integrals(norb, w.PES_SEED)
    h, g = w.pes_point(h0, h1, g0, w.PES_POINTS[10])
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    So = oracle.Sector.molecular(norb, norb // 2, norb // 2)
    psi = w.random_state(So.dim, 32)
    D, Dlo = So.dim, 12870
    rng = np.random.default_rng(32)
    rows = [0, 1, D - 2, D - 1]
    for r in (0, 1, 6434, 12868, 12869):           # first / last targets of some rows
        rows += [r * Dlo, r * Dlo + 1, r * Dlo + Dlo - 1]
        rows += [r * Dlo + 2047, r * Dlo + 2048, r * Dlo + 6 * 2048]  # column-tile edges (8 x 256 columns)
    rows = np.unique(np.concatenate([np.array(rows), rng.integers(0, D, 300)]))
    return h, g, R, So, psi, rows


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_apply_32_qubits_default_shape_sampled_rows(ps, mol32, dt):
    import torch
    h, g, R, So, psi, rows = mol32
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(16, 8, 8)
    assert S.dim == So.dim == 165636900
    ps.prepare(H, S)
    got = ps.launch_config(H, S, _tdt(dt))
    if dt == "c64":
        # the shape of the 32-qubit benchmarks: rank-staged rows, 8 columns per thread
        assert got["ranked"] == 1 and got["cols_per_thread"] == 8 and got["direct"] == 0, got
    xin = _rounded(psi, dt)
    x = torch.from_numpy(xin).to("cuda", _tdt(dt))
    out = ps.apply(H, S, x)
    torch.cuda.synchronize()
    sub = _gather(out, rows)
    del out
    ref = oracle_rows(So, R, xin, rows)
    assert _rel(sub, ref) <= TOL[dt]
    # the worst single row as well (no cancellation hides behind the norm)
    err = np.abs(sub - ref) / np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert err.max() <= 50 * TOL[dt]


# ----------------------------------------------------------------------------
# 64 batched molecules at full size
# ----------------------------------------------------------------------------
def test_batched_64_full_size_sampled_rows(ps):
    import torch
    mols = w.batched_states(64, 3)
    ints = [m.integrals() for m in mols]
    with cf.ThreadPoolExecutor(min(16, os.cpu_count() or 4)) as ex:
        Ros = list(ex.map(lambda hg_m: oracle.jw_hamiltonian(hg_m[1].norb, hg_m[0][0], hg_m[0][1], eps_drop=1e-12),
                          zip(ints, mols)))
    Hs = [ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12) for h, g in ints]
    Ss = [ps.Sector.molecular(m.norb, m.n_alpha, m.n_beta) for m in mols]
    psis = [w.random_state(S.dim, m.psi_seed).astype(np.complex64) for S, m in zip(Ss, mols)]
    x64 = [torch.from_numpy(p).to("cuda") for p in psis]
    outs = [torch.empty_like(x) for x in x64]
    B = ps.Batch(Hs, Ss, dtype=torch.complex64)
    tuned = B.tune(x64, outs, reps=1)
    rng = np.random.default_rng(64)
    samples = []
    for S in Ss:
        D = S.dim
        samples.append(np.unique(np.concatenate([[0, D - 1], rng.integers(0, D, 14)])))
    refs = []
    for b, m in enumerate(mols):
        So = oracle.Sector.molecular(m.norb, m.n_alpha, m.n_beta)
        refs.append(oracle_rows(So, Ros[b], psis[b].astype(np.complex128), samples[b]))
        del So
    shapes = [None, ps.LaunchConfig(cols_per_thread=0, staged_rows=1, row_split=1, direct=0, ranked=0, ms=0.0),
              ps.LaunchConfig(cols_per_thread=4, staged_rows=1, row_split=1, direct=0, ranked=1, ms=0.0),
              ps.LaunchConfig(cols_per_thread=4, staged_rows=1, row_split=1, direct=0, ranked=0, ms=0.0)]
    ran = []
    for shp in shapes:
        if shp is not None:
            B.set_launch_config(shp)
        ran.append(B.launch_config())
        for o in outs:
            o.fill_(float("nan"))
        res = B.apply(x64, outs).cpu().numpy()
        for b in range(64):
            sub = _gather(outs[b], samples[b])
            assert _rel(sub, refs[b]) <= TOL["c64"], (b, ran[-1])
            assert np.isfinite(res[b]).all()
    assert tuned["ms"] > 0 and {r["ranked"] for r in ran} == {0, 1}
    assert ran[1]["cols_per_thread"] == 0 and ran[1]["ms"] >= 2  # per-state shapes: one launch per shape group


# ----------------------------------------------------------------------------
# 24 qubits: 5% of the rows
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_24_qubits_five_percent_rows(ps, dt):
    import torch
    h, g = w.MOL24.integrals()
    R = oracle.jw_hamiltonian(12, h, g, eps_drop=1e-12)
    So = oracle.Sector.molecular(12, 6, 6)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(12, 6, 6)
    D, Dlo = S.dim, 924
    xin = _rounded(w.random_state(D, w.MOL24.psi_seed), dt)
    x = torch.from_numpy(xin).to("cuda", _tdt(dt))
    out = ps.apply(H, S, x)
    rng = np.random.default_rng(24)
    edges = np.concatenate([[r * Dlo, r * Dlo + Dlo - 1] for r in range(0, 924, 16)] + [[923 * Dlo + Dlo - 1]])
    rows = np.unique(np.concatenate([rng.choice(D, D // 20, replace=False), edges]))
    assert len(rows) >= D // 20
    sub = _gather(out, rows)
    ref = oracle_rows(So, R, xin, rows)
    assert _rel(sub, ref) <= TOL[dt]
