"""The SVD-factorised gather (launch shape direct = 4, eq. svd_sreverse_sum)
against the oracle: the factorisation's ranks against numpy's SVD of each
group's coefficient matrix built from the oracle's canonical terms (and the
paper's rank collapse: R_g <= 2 off the diagonal, R_0 = n_orb + 2), and H psi
element by element (1e-12 complex128, 1e-5 complex64, oracle on the rounded
input), including the 32-qubit sector whose tables run in several on-the-fly
batches."""
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


def _rounded(v, dt):
    return v if dt == "c128" else v.astype(np.complex64).astype(np.complex128)


def _ranks_numpy(R, n_lo):
    """Rank of every group's coefficient matrix over its distinct (z_lo, z_hi)
    masks, numpy SVD, singular values above 1e-12."""
    lomask = (1 << n_lo) - 1
    groups = {}
    for x, z, c in zip(R.x.tolist(), R.z.tolist(), R.c.tolist()):
        groups.setdefault(x, []).append((z & lomask, z >> n_lo, c.real))
    hist = np.zeros(65, np.int64)
    ranks = {}
    for x, terms in groups.items():
        a = sorted({t[0] for t in terms})
        b = sorted({t[1] for t in terms})
        M = np.zeros((len(a), len(b)))
        for za, zb, c in terms:
            M[a.index(za), b.index(zb)] += c
        r = int(np.sum(np.linalg.svd(M, compute_uv=False) > 1e-12))
        hist[r] += 1
        ranks[x] = r
    return hist, ranks


@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (8, 4, 4), (10, 5, 5)])
def test_svd_ranks_match_numpy_and_the_rank_collapse(ps, norb, na, nb):
    h, g = w.molecular_integrals(norb, 0)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, na, nb)
    hist, nbatch = ps.svd_ranks(H, S)
    ref, ranks = _ranks_numpy(R, norb)
    assert np.array_equal(hist[:65], ref[:65])
    assert nbatch == 1
    assert ranks[0] == norb + 2
    assert max(r for x, r in ranks.items() if x != 0) <= 2


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (8, 4, 4), (7, 2, 5), (10, 5, 5), (5, 0, 2)])
def test_svd_gather_matches_oracle(ps, dt, norb, na, nb):
    import torch
    h, g = w.molecular_integrals(norb, 1)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, na, nb)
    So = oracle.Sector.molecular(norb, na, nb)
    psi = _rounded(w.random_state(S.dim, 40 + norb), dt)
    ref = oracle.apply(So, R, psi)
    E = oracle.expect(So, R, psi)[0]
    ps.prepare(H, S)
    x = torch.from_numpy(psi).to("cuda", _tdt(dt))
    for tpt in (1, 2, 4):
        ps.set_launch_config(H, S, _tdt(dt), ps.LaunchConfig(cols_per_thread=tpt, staged_rows=1, row_split=1,
                                                             direct=4, ranked=1, ms=0.0))
        got = ps.launch_config(H, S, _tdt(dt))
        assert got["direct"] == 4 and got["cols_per_thread"] == tpt, got
        out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
        scale = max(np.linalg.norm(ref), 1e-3 * np.abs(R.c).sum())
        assert np.linalg.norm(out - ref) <= TOL[dt] * scale, tpt
        r = ps.expect(H, S, x).cpu().numpy()
        assert abs(complex(r[0], r[1]) - E) <= (1e-12 if dt == "c128" else 1e-6) * max(1.0, abs(E)), tpt


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_svd_gather_24_qubits(ps, dt):
    import torch
    from test_gpu_parity_shapes import oracle_rows
    h, g = w.MOL24.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(12, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(12, 6, 6)
    So = oracle.Sector.molecular(12, 6, 6)
    ps.prepare(H, S)
    ps.set_launch_config(H, S, _tdt(dt), ps.LaunchConfig(cols_per_thread=1, staged_rows=1, row_split=1, direct=4,
                                                         ranked=1, ms=0.0))
    psi = _rounded(w.random_state(S.dim, w.MOL24.psi_seed), dt)
    x = torch.from_numpy(psi).to("cuda", _tdt(dt))
    out = ps.apply(H, S, x)
    rows = np.unique(np.concatenate([np.random.default_rng(7).choice(S.dim, 20000, replace=False),
                                     [0, 923, 924, S.dim - 1]]))
    idx = torch.from_numpy(rows).to("cuda")
    sub = out.index_select(0, idx).cpu().numpy().astype(np.complex128)
    ref = oracle_rows(So, R, psi, rows)
    assert np.linalg.norm(sub - ref) <= TOL[dt] * np.linalg.norm(ref)
    # the same vector as the default (popcount) gather
    ps.set_launch_config(H, S, _tdt(dt), ps.LaunchConfig(cols_per_thread=4, staged_rows=1, row_split=1, direct=0,
                                                         ranked=0, ms=0.0))
    base = ps.apply(H, S, x)
    d = torch.linalg.vector_norm((out - base).to(torch.complex128)).item()
    assert d <= 2 * TOL[dt] * torch.linalg.vector_norm(base.to(torch.complex128)).item()


def test_svd_gather_32_qubits_batches(ps):
    """16 orbitals: the alpha tables run in several on-the-fly batches (later
    batches add to the output); sampled rows against the oracle, and an
    expectation without an output vector is refused."""
    import torch
    from test_gpu_parity_shapes import oracle_rows
    norb = 16
    h0, h1, g0 = w.pes_integrals(norb, w.PES_SEED)
    h, g = w.pes_point(h0, h1, g0, w.PES_POINTS[10])
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, 8, 8)
    So = oracle.Sector.molecular(norb, 8, 8)
    hist, nbatch = ps.svd_ranks(H, S)
    assert nbatch > 1 and hist[norb + 2] >= 1 and hist[3:norb + 2].sum() == 0
    ps.prepare(H, S)
    ps.set_launch_config(H, S, torch.complex64, ps.LaunchConfig(cols_per_thread=2, staged_rows=1, row_split=1,
                                                                direct=4, ranked=1, ms=0.0))
    psi = _rounded(w.random_state(S.dim, 33), "c64")
    x = torch.from_numpy(psi).to("cuda", torch.complex64)
    out = ps.apply(H, S, x)
    rows = np.unique(np.concatenate([np.random.default_rng(3).integers(0, S.dim, 300), [0, S.dim - 1]]))
    idx = torch.from_numpy(rows).to("cuda")
    sub = out.index_select(0, idx).cpu().numpy().astype(np.complex128)
    ref = oracle_rows(So, R, psi, rows)
    assert np.linalg.norm(sub - ref) <= TOL["c64"] * np.linalg.norm(ref)
    with pytest.raises(ps.PauliError) as e:
        ps.expect(H, S, x)
    assert e.value.code == ps.EUNSUPPORTED
    hp = torch.empty_like(x)
    r = ps.expect(H, S, x, hpsi_out=hp).cpu().numpy()
    assert np.isfinite(r).all()


def test_svd_needs_a_real_operator(ps):
    n = 8
    H = ps.PauliSum.from_terms(n, [0b11], [0b01], [1.0], [0.5], form=ps.XZ)  # complex coefficient
    S = ps.Sector.molecular(4, 2, 2)
    with pytest.raises(ps.PauliError) as e:
        ps.svd_ranks(H, S)
    assert e.value.code == ps.EUNSUPPORTED
