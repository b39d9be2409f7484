"""GPU apply / expect / rotate vs the oracle on the same seeded inputs.

Tolerances: ||H psi||-relative error <= 1e-12 for the
FP64 (complex128) path and <= 1e-5 for the FP32 (complex64) path, the latter
measured against the oracle run on the complex64-rounded input; energies within
1e-6 Ha (1e-12 for FP64)."""
import math

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


def _to_dev(psi, name):
    import torch
    return torch.from_numpy(np.ascontiguousarray(psi)).to("cuda", _tdt(name))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _mol(norb, na, nb, seed=0, eps=1e-12):
    h, g = w.molecular_integrals(norb, seed)
    return h, g, oracle.jw_hamiltonian(norb, h, g, eps_drop=eps)


# ----------------------------------------------------------------------------
# apply, whole vectors
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (8, 4, 4), (7, 2, 5), (10, 5, 5)])
def test_apply_molecular_sector(ps, dt, norb, na, nb):
    h, g, R = _mol(norb, na, nb)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, na, nb)
    So = oracle.Sector.molecular(norb, na, nb)
    psi = w.random_state(S.dim, 100 + norb)
    x = _to_dev(psi, dt)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))
    assert _rel(out, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("n,n_lo", [(8, 0), (12, 5), (13, 10)])
def test_apply_full_space_complex_sum(ps, dt, n, n_lo):
    """Non-Hermitian complex Pauli sum (complex-coefficient path), full 2^n space."""
    x_, z_, gamma, cre, cim = w.random_pauli_terms(n, 300, 5 + n, dup_frac=0.2)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim, gamma=gamma)
    R = oracle.build_sum(n, x_, z_, gamma, cre, cim)
    S = ps.Sector.full(n, n_lo)
    So = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 9)
    x = _to_dev(psi, dt)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))
    assert _rel(out, ref) <= TOL[dt]


def _diag_rich_terms(n, seed):
    """Complex sum with a large x = 0 group (Z strings on low-only, high-only and
    crossing bit sets, the identity) and a few off-diagonal groups."""
    rng = np.random.default_rng(seed)
    xs, zs, cre, cim = [0], [0], [0.7], [0.0]
    for _ in range(120):
        xs.append(0)
        zs.append(int(rng.integers(1, 1 << n)))
        cre.append(rng.normal())
        cim.append(0.3 * rng.normal())
    for _ in range(20):
        xm = int(rng.integers(1, 1 << n))
        for _ in range(3):
            xs.append(xm)
            zs.append(int(rng.integers(0, 1 << n)))
            cre.append(rng.normal())
            cim.append(rng.normal())
    return (np.array(xs, np.uint64), np.array(zs, np.uint64), np.array(cre), np.array(cim))


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("n_lo", [5, 10, 12, 13])
def test_apply_direct_diagonal_table(ps, dt, n_lo):
    """The small-operator (direct) gather with the x = 0 group's z_hi = 0 part
    tabulated over the low bits (n_lo <= 12) and without (13), against the
    oracle and against the staged gather."""
    n = 15
    x_, z_, cre, cim = _diag_rich_terms(n, 40 + n_lo)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim, form=ps.XZ)
    R = oracle.build_sum(n, x_, z_, None, cre, cim, letter_form=False)
    S = ps.Sector.full(n, n_lo)
    So = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 17)
    x = _to_dev(psi, dt)
    ref = oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))
    outs = []
    for direct in (1, 0):
        ps.prepare(H, S)
        c = ps.LaunchConfig(cols_per_thread=4 if direct else 1, staged_rows=1, row_split=1, direct=direct, ranked=0,
                            ms=0.0)
        ps.set_launch_config(H, S, _tdt(dt), c)
        out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
        assert _rel(out, ref) <= TOL[dt], direct
        outs.append(out)
        r = ps.expect(H, S, x).cpu().numpy()
        e_ref = np.vdot(x.cpu().numpy().astype(np.complex128), ref)
        assert abs(complex(r[0], r[1]) - e_ref) <= TOL[dt] * np.linalg.norm(ref) * np.linalg.norm(psi)


def _lattice_terms(n, seed):
    """Complex sum of short-range groups (bit pairs at distance 1..3, 2-4 terms with
    z anywhere) and a diagonal group of 50 random Z strings."""
    rng = np.random.default_rng(seed)
    xs, zs, cre, cim = [], [], [], []
    for _ in range(50):
        xs.append(0)
        zs.append(int(rng.integers(1, 1 << n)))
        cre.append(rng.normal())
        cim.append(0.2 * rng.normal())
    for a, d in zip(rng.integers(0, n - 1, 30), rng.integers(1, 4, 30)):
        xm = (1 << int(a)) | (1 << min(int(a) + int(d), n - 1))
        for _ in range(int(rng.integers(2, 5))):
            xs.append(xm)
            zs.append(int(rng.integers(0, 1 << n)))
            cre.append(rng.normal())
            cim.append(rng.normal())
    return (np.array(xs, np.uint64), np.array(zs, np.uint64), np.array(cre), np.array(cim))


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("case", ["xxz16", "lattice17"])
@pytest.mark.parametrize("tpt", [1, 8])
def test_apply_local_passes(ps, dt, case, tpt):
    """The full space in passes over local bit sets (2 passes here, forced at this
    size), 4 targets per thread (cols_per_thread 1: the default) or 8: apply and
    expect against the oracle, with and without the H psi output."""
    import torch
    if case == "xxz16":
        n = 16
        x_, z_, cre, cim = w.xxz_terms(n, 1)
        H = ps.PauliSum.from_terms(n, x_, z_, cre, cim)
        R = oracle.build_sum(n, x_, z_, None, cre, cim)
    else:
        n = 17
        x_, z_, cre, cim = _lattice_terms(n, 5)
        H = ps.PauliSum.from_terms(n, x_, z_, cre, cim, form=ps.XZ)
        R = oracle.build_sum(n, x_, z_, None, cre, cim, letter_form=False)
    S = ps.Sector.full(n)
    So = oracle.Sector.full(n)
    ps.prepare(H, S)
    c = ps.LaunchConfig(cols_per_thread=tpt, staged_rows=1, row_split=1, direct=2, ranked=0, ms=0.0)
    ps.set_launch_config(H, S, _tdt(dt), c)
    got = ps.launch_config(H, S, _tdt(dt))
    assert got["direct"] == 2 and got["cols_per_thread"] == (8 if tpt == 8 else 4), got
    psi = w.random_state(1 << n, 23)
    x = _to_dev(psi, dt)
    xin = x.cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, xin)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    assert _rel(out, ref) <= TOL[dt]
    e_ref = np.vdot(xin, ref)
    for hp in (None, torch.empty_like(x)):
        r = ps.expect(H, S, x, hpsi_out=hp).cpu().numpy()
        assert abs(complex(r[0], r[1]) - e_ref) <= TOL[dt] * np.linalg.norm(ref) * np.linalg.norm(xin)
        assert abs(r[2] - np.linalg.norm(ref) ** 2) <= 10 * TOL[dt] * np.linalg.norm(ref) ** 2
        if hp is not None:
            assert _rel(hp.cpu().numpy().astype(np.complex128), ref) <= TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("case", ["xxz17", "lattice18"])
def test_apply_local_cluster_passes(ps, dt, case):
    """Windows of 16 bits shared by clusters of 8 CTAs (X masks on the cluster bits
    read a peer's chunk through distributed shared memory), forced with
    ranked = 1: apply and expect against the oracle."""
    import torch
    if case == "xxz17":
        n = 17
        x_, z_, cre, cim = w.xxz_terms(n, 1)
        H = ps.PauliSum.from_terms(n, x_, z_, cre, cim)
        R = oracle.build_sum(n, x_, z_, None, cre, cim)
    else:
        n = 18
        x_, z_, cre, cim = _lattice_terms(n, 7)
        H = ps.PauliSum.from_terms(n, x_, z_, cre, cim, form=ps.XZ)
        R = oracle.build_sum(n, x_, z_, None, cre, cim, letter_form=False)
    S = ps.Sector.full(n)
    So = oracle.Sector.full(n)
    ps.prepare(H, S)
    c = ps.LaunchConfig(cols_per_thread=1, staged_rows=1, row_split=1, direct=2, ranked=1, ms=0.0)
    ps.set_launch_config(H, S, _tdt(dt), c)
    got = ps.launch_config(H, S, _tdt(dt))
    assert got["direct"] == 2 and got["ranked"] == 1, got
    psi = w.random_state(1 << n, 31)
    x = _to_dev(psi, dt)
    xin = x.cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, xin)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    assert _rel(out, ref) <= TOL[dt]
    e_ref = np.vdot(xin, ref)
    for hp in (None, torch.empty_like(x)):
        r = ps.expect(H, S, x, hpsi_out=hp).cpu().numpy()
        assert abs(complex(r[0], r[1]) - e_ref) <= TOL[dt] * np.linalg.norm(ref) * np.linalg.norm(xin)
        if hp is not None:
            assert _rel(hp.cpu().numpy().astype(np.complex128), ref) <= TOL[dt]
    # the unclustered passes give the same vector
    ps.set_launch_config(H, S, _tdt(dt), ps.LaunchConfig(cols_per_thread=1, staged_rows=1, row_split=1, direct=2,
                                                         ranked=0, ms=0.0))
    assert ps.launch_config(H, S, _tdt(dt))["ranked"] == 0
    out2 = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    assert _rel(out2, out) <= 2 * TOL[dt]


def test_apply_local_cluster_27_sites(ps):
    """At 27 sites the clustered windows need 2 passes where 13-bit chunks need 3
    (installed with ranked = 1; the plain passes stay the default); sampled rows
    against the per-row oracle."""
    import torch
    n = 27
    x_, z_, cre, cim = w.xxz_terms(n, 1)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim)
    R = oracle.build_sum(n, x_, z_, None, cre, cim)
    S = ps.Sector.full(n)
    So = oracle.Sector.full(n)
    ps.prepare(H, S)
    assert ps.launch_config(H, S)["ranked"] == 0
    ps.set_launch_config(H, S, torch.complex64, ps.LaunchConfig(cols_per_thread=4, staged_rows=1, row_split=1,
                                                                direct=2, ranked=1, ms=0.0))
    psi = w.random_state(1 << n, 37)
    x = _to_dev(psi, "c64")
    out = ps.apply(H, S, x)
    cfg = ps.launch_config(H, S)
    assert cfg["direct"] == 2 and cfg["ranked"] == 1, cfg
    rows = np.random.default_rng(2).integers(0, 1 << n, 300)
    rows = np.concatenate([rows, [0, 1, 7, 8, (1 << 16) - 1, 1 << 16, (1 << n) - 1]])
    ref = oracle.apply_rows(So, R, x.cpu().numpy().astype(np.complex128), rows)
    got = out.cpu().numpy().astype(np.complex128)[rows]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, scale) * 10


def test_apply_local_passes_24_sites_default(ps):
    """At 24 sites the pass scheme is the default launch of the full space (3 passes
    for the open chain); sampled rows against the per-row oracle."""
    n = 24
    x_, z_, cre, cim = w.xxz_terms(n, 1)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim)
    R = oracle.build_sum(n, x_, z_, None, cre, cim)
    S = ps.Sector.full(n)
    So = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 29)
    x = _to_dev(psi, "c64")
    out = ps.apply(H, S, x)
    assert ps.launch_config(H, S)["direct"] == 2
    rows = np.random.default_rng(1).integers(0, 1 << n, 300)
    rows = np.concatenate([rows, [0, 1, 7, 8, (1 << n) - 1]])
    ref = oracle.apply_rows(So, R, x.cpu().numpy().astype(np.complex128), rows)
    got = out.cpu().numpy().astype(np.complex128)[rows]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, scale) * 10


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_multiblock_sz0_xxz(ps, dt):
    """Open XXZ chain, 14 sites, Sz = 0 as 8 product blocks (k, 7-k) of a 7|7 split."""
    n = 14
    x_, z_, cre, cim = w.xxz_terms(n, 1)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim)
    R = oracle.build_sum(n, x_, z_, None, cre, cim)
    blocks = [(k, 7 - k) for k in range(8)]
    S = ps.Sector(n, ps.BLOCKS, 7, blocks)
    So = oracle.Sector(n, oracle.BLOCKS, 7, blocks)
    psi = w.random_state(S.dim, 21)
    x = _to_dev(psi, dt)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))
    assert _rel(out, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb", [(16, 1, 1), (16, 2, 1), (15, 2, 2), (14, 2, 1)])
def test_apply_wide_split_rank_staged(ps, dt, norb, na, nb):
    """Low half of 14-16 qubits: rows staged densely by rank (full u16 rank table
    up to 14 bits, byte-split tables above)."""
    h, g = w.molecular_integrals(norb, 2)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, na, nb)
    So = oracle.Sector.molecular(norb, na, nb)
    psi = w.random_state(S.dim, 5)
    x = _to_dev(psi, dt)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))
    assert _rel(out, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_rank_staged_matches_pattern_staged(ps, dt):
    """The two staging layouts (forced through the launch-shape interface) agree with the oracle."""
    import torch
    h, g, R = _mol(8, 4, 4)
    S = ps.Sector.molecular(8, 4, 4)
    So = oracle.Sector.molecular(8, 4, 4)
    psi = w.random_state(S.dim, 12)
    code = ps.C64 if dt == "c64" else ps.C128
    for ranked in (0, 1):
        H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
        ps.prepare(H, S)
        c = ps.LaunchConfig(cols_per_thread=1, staged_rows=1, row_split=2, direct=0, ranked=ranked, ms=0.0)
        ps._check(ps.lib().pauli_set_launch_config(H._h, S._h, code, ps.C.byref(c)))
        assert ps.launch_config(H, S, torch.complex64 if dt == "c64" else torch.complex128)["ranked"] == ranked
        x = _to_dev(psi, dt)
        out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
        assert _rel(out, oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))) <= TOL[dt]
        r = ps.expect(H, S, x).cpu().numpy()
        E, _ = oracle.expect(So, R, x.cpu().numpy().astype(np.complex128))
        assert abs(complex(r[0], r[1]) - E) <= (1e-12 if dt == "c128" else 1e-6)


def _force_list(ps, H, S, dt, split):
    """Install the list-driven gather (direct = 3) with the given row split."""
    ps.prepare(H, S)
    c = ps.LaunchConfig(cols_per_thread=1, staged_rows=1, row_split=split, direct=3, ranked=0, ms=0.0)
    ps.set_launch_config(H, S, _tdt(dt), c)
    cfg = ps.launch_config(H, S, _tdt(dt))
    # the split is capped at one range per eight pieces of the plan
    assert cfg["direct"] == 3 and 1 <= cfg["row_split"] <= split, cfg


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb,split", [(6, 3, 3, 1), (8, 4, 4, 2), (7, 2, 5, 1), (10, 5, 5, 4),
                                              (4, 0, 2, 1), (4, 4, 1, 2)])
def test_apply_list_gather_molecular(ps, dt, norb, na, nb, split):
    """The gather over per-item lists of valid (target, source) pairs, forced on
    single-block sectors (including one-configuration low halves, k_lo = 0 and
    k_lo = n_lo), against the oracle for apply and expect."""
    h, g, R = _mol(norb, na, nb)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, na, nb)
    So = oracle.Sector.molecular(norb, na, nb)
    _force_list(ps, H, S, dt, split)
    x = _to_dev(w.random_state(S.dim, 200 + norb), dt)
    xin = x.cpu().numpy().astype(np.complex128)
    ref = oracle.apply(So, R, xin)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    scale = max(np.linalg.norm(ref), 1e-3 * np.abs(R.c).sum())
    assert np.linalg.norm(out - ref) <= TOL[dt] * scale
    r = ps.expect(H, S, x).cpu().numpy()
    E, _ = oracle.expect(So, R, xin)
    assert abs(complex(r[0], r[1]) - E) <= (1e-12 if dt == "c128" else 1e-6) * max(1.0, np.abs(R.c).sum())
    assert abs(r[2] - np.vdot(ref, ref).real) <= 10 * TOL[dt] * max(np.vdot(ref, ref).real, 1e-6)


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("n,n_lo,blk,split", [(12, 6, (3, 3), 1), (16, 8, (4, 4), 2), (16, 10, (5, 3), 1)])
def test_apply_list_gather_complex_sum(ps, dt, n, n_lo, blk, split):
    """Complex coefficients (the non-real path) and X masks that leave the block:
    items whose x_lo has odd popcount have empty lists."""
    x_, z_, gam, cre, cim = w.random_pauli_terms(n, 300, 31 + n_lo)
    H = ps.PauliSum.from_terms(n, x_, z_, cre, cim, gamma=gam)
    R = oracle.build_sum(n, x_, z_, gam, cre, cim)
    S = ps.Sector(n, ps.BLOCKS, n_lo, [blk])
    So = oracle.Sector(n, oracle.BLOCKS, n_lo, [blk])
    _force_list(ps, H, S, dt, split)
    x = _to_dev(w.random_state(S.dim, 77), dt)
    ref = oracle.apply(So, R, x.cpu().numpy().astype(np.complex128))
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    assert _rel(out, ref) <= TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_list_gather_24_qubits(ps, mol24, dt):
    """The list gather without a split at full size: sampled rows against the
    oracle, and the whole vector against the staged gather."""
    h, g, H, R, S, So, psi = mol24
    x = _to_dev(psi, dt)
    xin = x.cpu().numpy().astype(np.complex128)
    H2 = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    _force_list(ps, H2, S, dt, 1)
    out = ps.apply(H2, S, x).cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(6)
    rows = np.unique(np.concatenate([rng.integers(0, S.dim, 150), [0, 923, 924, S.dim - 1]]))
    ref = oracle.apply_rows(So, R, xin, rows)
    assert np.linalg.norm(out[rows] - ref) <= TOL[dt] * 1.5 * np.linalg.norm(ref)
    H3 = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    ps.prepare(H3, S)
    c = ps.LaunchConfig(cols_per_thread=4, staged_rows=1, row_split=4, direct=0, ranked=0, ms=0.0)
    ps.set_launch_config(H3, S, _tdt(dt), c)
    staged = ps.apply(H3, S, x).cpu().numpy().astype(np.complex128)
    assert _rel(out, staged) <= 2 * TOL[dt]


def test_apply_edge_cases(ps):
    import torch
    # empty operator -> zero vector
    H0 = ps.PauliSum.from_terms(6, [], [], [])
    S = ps.Sector.molecular(3, 1, 2)
    x = _to_dev(w.random_state(S.dim, 1), "c128")
    assert torch.count_nonzero(ps.apply(H0, S, x)).item() == 0
    # one-configuration sectors (k = 0 and k = n) and a diagonal-only operator
    h, g = w.molecular_integrals(4, 3)
    H = ps.PauliSum.jw_molecular(h, g)
    R = oracle.jw_hamiltonian(4, h, g)
    for na, nb in [(0, 0), (4, 4), (0, 4), (1, 0)]:
        S = ps.Sector.molecular(4, na, nb)
        So = oracle.Sector.molecular(4, na, nb)
        psi = w.random_state(S.dim, 2)
        out = ps.apply(H, S, _to_dev(psi, "c128")).cpu().numpy()
        ref = oracle.apply(So, R, psi)
        # the vacuum row is pure rounding noise of cancelling terms: bound by the operator scale
        assert np.linalg.norm(out - ref) <= 1e-12 * max(np.linalg.norm(ref), np.abs(R.c).sum())
    # in-place (aliased) apply is rejected
    S = ps.Sector.molecular(4, 2, 2)
    y = _to_dev(w.random_state(S.dim, 3), "c128")
    with pytest.raises(ps.PauliError):
        ps.apply(H, S, y, y)


# ----------------------------------------------------------------------------
# full-size workload: 24 qubits, (6a,6b), D = 853,776 -- sampled rows + properties
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def mol24(ps):
    h, g = w.MOL24.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(12, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(12, 6, 6)
    So = oracle.Sector.molecular(12, 6, 6)
    psi = w.random_state(S.dim, w.MOL24.psi_seed)
    return h, g, H, R, S, So, psi


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_24_qubits_sampled_rows(ps, mol24, dt):
    h, g, H, R, S, So, psi = mol24
    x = _to_dev(psi, dt)
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    xin = x.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(5)
    D = S.dim
    rows = np.unique(np.concatenate([rng.integers(0, D, 200), [0, 1, 923, 924, 925, D - 925, D - 2, D - 1]]))
    ref = oracle.apply_rows(So, R, xin, rows)
    assert np.linalg.norm(out[rows] - ref) <= TOL[dt] * 1.5 * np.linalg.norm(ref)


def test_apply_24_qubits_properties(ps, mol24):
    """Hermiticity <phi|H psi> = conj <psi|H phi> and c64 vs c128 agreement at full size."""
    h, g, H, R, S, So, psi = mol24
    phi = w.random_state(S.dim, 99)
    a = ps.apply(H, S, _to_dev(psi, "c128")).cpu().numpy()
    b = ps.apply(H, S, _to_dev(phi, "c128")).cpu().numpy()
    assert abs(np.vdot(phi, a) - np.conj(np.vdot(psi, b))) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b) * 10
    a32 = ps.apply(H, S, _to_dev(psi, "c64")).cpu().numpy().astype(np.complex128)
    assert _rel(a32, a) <= 1e-5


# ----------------------------------------------------------------------------
# expectation values
# ----------------------------------------------------------------------------
def test_expect_both_precisions_on_one_plan(ps):
    """13 orbitals, (6a,6b): the complex64 launch splits its rows while the
    complex128 one does not, so the plan's partial sums must be sized for both
    (complex128 first, then complex64, then again); the two energies agree."""
    import torch
    norb = 13
    h, g = w.molecular_integrals(norb, 4)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, 6, 6)
    psi = w.random_state(S.dim, 77)
    x128 = _to_dev(psi, "c128")
    x64 = _to_dev(psi, "c64")
    ps.prepare(H, S)
    cfg64, cfg128 = ps.launch_config(H, S, torch.complex64), ps.launch_config(H, S, torch.complex128)
    assert cfg64["row_split"] > 1 and cfg128["row_split"] == 1
    e = []
    for x in (x128, x64, x128, x64):
        r = ps.expect(H, S, x, hpsi_out=torch.empty_like(x)).cpu().numpy()
        e.append(r[0])
    assert abs(e[0] - e[2]) == 0.0 and abs(e[1] - e[3]) == 0.0  # fixed reduction order
    assert abs(e[0] - e[1]) <= 1e-6 * max(1.0, abs(e[0]))


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_expect_matches_oracle_and_hf(ps, dt):
    h, g, R = _mol(6, 3, 3)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(6, 3, 3)
    So = oracle.Sector.molecular(6, 3, 3)
    psi = w.random_state(S.dim, 11)
    x = _to_dev(psi, dt)
    hp = _to_dev(np.zeros(S.dim, complex), dt)
    res = ps.expect(H, S, x, hpsi_out=hp).cpu().numpy()
    xin = x.cpu().numpy().astype(np.complex128)
    E, n2 = oracle.expect(So, R, xin)
    assert abs(complex(res[0], res[1]) - E) <= (1e-12 if dt == "c128" else 1e-6)
    assert abs(res[2] - n2) <= (1e-11 if dt == "c128" else 1e-5) * n2
    assert abs(res[3] - np.vdot(xin, xin).real) <= 1e-12
    assert _rel(hp.cpu().numpy().astype(np.complex128), oracle.apply(So, R, xin)) <= TOL[dt]
    # Hartree-Fock determinant: closed form
    hf = np.zeros(S.dim, complex)
    hf[So.index(oracle.hf_config(6, 3, 3))[0]] = 1.0
    r = ps.expect(H, S, _to_dev(hf, dt)).cpu().numpy()
    assert abs(r[0] - oracle.hf_energy(6, h, g, 3, 3)) <= (1e-12 if dt == "c128" else 1e-6)


def test_expect_24_qubits(ps, mol24):
    h, g, H, R, S, So, psi = mol24
    hf = np.zeros(S.dim, complex)
    hf[So.index(oracle.hf_config(12, 6, 6))[0]] = 1.0
    e_hf = oracle.hf_energy(12, h, g, 6, 6)
    for dt, tol in (("c128", 1e-12), ("c64", 1e-6)):
        r = ps.expect(H, S, _to_dev(hf, dt)).cpu().numpy()
        assert abs(r[0] - e_hf) <= tol
    r128 = ps.expect(H, S, _to_dev(psi, "c128")).cpu().numpy()
    r64 = ps.expect(H, S, _to_dev(psi, "c64")).cpu().numpy()
    assert abs(r128[0] - r64[0]) <= 1e-6
    assert abs(r128[1]) <= 1e-12


def test_expect_is_deterministic(ps, mol24):
    h, g, H, R, S, So, psi = mol24
    x = _to_dev(psi, "c64")
    a = ps.expect(H, S, x).cpu().numpy()
    b = ps.expect(H, S, x).cpu().numpy()
    assert np.array_equal(a, b)


# ----------------------------------------------------------------------------
# rotation
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_rotate_pair_double_and_group(ps, dt):
    norb = 6
    S = ps.Sector.molecular(norb, 3, 3)
    So = oracle.Sector.molecular(norb, 3, 3)
    h, g, R = _mol(norb, 3, 3)
    xs, cnt = np.unique(R.x, return_counts=True)
    gx = xs[np.argmax(cnt * (xs != 0))]
    sel = R.x == gx
    grp = oracle.PauliSum(12, R.x[sel], R.z[sel], R.c[sel])
    cases = [(ps.PauliSum.jw_fermion(12, w.pair_double_generator(norb, 0, 4)),
              oracle.fermion_sum(12, w.pair_double_generator(norb, 0, 4))),
             (ps.PauliSum.from_terms(12, grp.x, grp.z, grp.c.real, grp.c.imag, form=ps.XZ), grp)]
    for G, Go in cases:
        psi = w.random_state(S.dim, 31)
        for theta in (0.41, -1.7):
            x = _to_dev(psi, dt)
            xin = x.cpu().numpy().astype(np.complex128)
            ps.rotate(G, S, theta, x)
            ref = oracle.rotate(So, Go, theta, xin)
            assert _rel(x.cpu().numpy().astype(np.complex128), ref) <= TOL[dt]
        assert G.status() == ps.OK


def test_rotate_single_string_full_space(ps):
    n = 9
    P = ps.PauliSum.from_terms(n, [0b100101], [0b001100], [1.0])  # letters X0 Y2 Z3 X5
    Po = oracle.build_sum(n, np.array([0b100101], np.uint64), np.array([0b001100], np.uint64), None,
                          np.array([1.0]), np.array([0.0]))
    S = ps.Sector.full(n)
    So = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 4)
    Ppsi = oracle.apply(So, Po, psi)
    for theta in (0.3, math.pi / 2):
        x = _to_dev(psi, "c128")
        ps.rotate(P, S, theta, x)
        ref = math.cos(theta) * psi - 1j * math.sin(theta) * Ppsi
        assert _rel(x.cpu().numpy(), ref) <= 1e-13


def test_rotate_diagonal_group(ps):
    n = 8
    zs = np.array([0b1, 0b110, 0b10010000], np.uint64)
    P = ps.PauliSum.from_terms(n, np.zeros(3, np.uint64), zs, [0.3, -0.7, 0.25])
    Po = oracle.build_sum(n, np.zeros(3, np.uint64), zs, None, np.array([0.3, -0.7, 0.25]), np.zeros(3))
    S = ps.Sector.full(n)
    So = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 5)
    x = _to_dev(psi, "c128")
    ps.rotate(P, S, 0.9, x)
    assert _rel(x.cpu().numpy(), oracle.rotate(So, Po, 0.9, psi)) <= 1e-12


def test_rotate_errors(ps):
    norb = 4
    S = ps.Sector.molecular(norb, 2, 2)
    Go = oracle.fermion_sum(8, w.pair_double_generator(norb, 0, 2))
    # one JW string of a pair double leaks out of the sector: device status PAULI_ESECTOR
    one = ps.PauliSum.from_terms(8, Go.x[:1], Go.z[:1], Go.c[:1].real, Go.c[:1].imag, form=ps.XZ)
    x = _to_dev(w.random_state(S.dim, 6), "c128")
    ps.rotate(one, S, 0.3, x)
    assert one.status() == ps.ESECTOR
    assert one.status() == ps.OK  # reading clears the word
    # two X masks
    two = ps.PauliSum.from_terms(8, [3, 5], [0, 0], [1.0, 1.0])
    with pytest.raises(ps.PauliError) as e:
        ps.rotate(two, S, 0.3, x)
    assert e.value.code == ps.EINVAL
    # non-Hermitian generator
    nh = ps.PauliSum.from_terms(8, [3], [0], [0.0], [1.0])
    with pytest.raises(ps.PauliError) as e:
        ps.rotate(nh, ps.Sector.full(8), 0.3, _to_dev(w.random_state(256, 1), "c128"))
    assert e.value.code == ps.ENOTHERMITIAN
