"""GPU build path vs oracle: Jordan-Wigner raw entries, canonical reduction, groups and
sector rank / unrank -- all bit-exact (integer and exact-sum work)."""
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


def _same(a, b):
    """Exact equality (== on floats: bit-exact up to the sign of zero)."""
    return a.shape == b.shape and np.array_equal(a, b)


@pytest.mark.parametrize("norb,seed,e_nn", [(3, 1, 0.0), (6, 0, 0.0), (6, 0, 1.5)])
def test_jw_raw_entries_bit_exact(ps, norb, seed, e_nn):
    h, g = w.molecular_integrals(norb, seed)
    gx, gz, gc = ps.jw_molecular_raw(h, g, e_nn=e_nn)
    ox, oz, oc = oracle.jw_raw(norb, h, g)
    if e_nn != 0.0:
        ox = np.concatenate([[0], ox]).astype(np.uint64)
        oz = np.concatenate([[0], oz]).astype(np.uint64)
        oc = np.concatenate([[e_nn], oc])
    assert _same(gx, ox) and _same(gz, oz) and _same(gc, oc)


@pytest.mark.parametrize("norb,eps_drop", [(6, 0.0), (6, 1e-12), (8, 1e-12), (12, 1e-12)])
def test_jw_hamiltonian_canonical_bit_exact(ps, norb, eps_drop):
    h, g = w.molecular_integrals(norb, 0)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=eps_drop)
    x, z, c = H.export()
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=eps_drop)
    assert _same(x, R.x) and _same(z, R.z) and _same(c, R.c)
    gx, gs = H.groups()
    ux, first = np.unique(R.x, return_index=True)
    assert _same(gx, ux) and _same(gs, np.concatenate([first, [R.m]]).astype(np.int64))


def test_eps_int_threshold_bit_exact(ps):
    h, g = w.molecular_integrals(5, 9)
    H = ps.PauliSum.jw_molecular(h, g, eps_int=0.05, eps_drop=0.0)
    R = oracle.jw_hamiltonian(5, h, g, eps_int=0.05)
    x, z, c = H.export()
    assert _same(x, R.x) and _same(z, R.z) and _same(c, R.c)


@pytest.mark.parametrize("n,m,eps,form", [(3, 50, 0.0, 0), (24, 5000, 0.0, 0), (64, 3000, 0.5, 1),
                                          (40, 20000, 1e-3, 0), (1, 7, 0.0, 1)])
def test_sum_build_canonical_bit_exact(ps, n, m, eps, form):
    x, z, gamma, cre, cim = w.random_pauli_terms(n, m, 77 + n, dup_frac=0.5)
    H = ps.PauliSum.from_terms(n, x, z, cre, cim, gamma=gamma, form=form, eps_drop=eps)
    R = oracle.build_sum(n, x, z, gamma, cre, cim, eps=eps, letter_form=(form == 0))
    gx_, gz_, gc_ = H.export()
    assert _same(gx_, R.x) and _same(gz_, R.z) and _same(gc_, R.c)


def test_sum_build_empty_and_cancelling(ps):
    H = ps.PauliSum.from_terms(4, [], [], [])
    assert H.info() == (4, 0, 0)
    H2 = ps.PauliSum.from_terms(4, [3, 3], [1, 1], [0.25, -0.25], form=1)
    assert H2.m == 0 and H2.n_groups == 0


def test_fermion_terms_bit_exact(ps):
    terms = w.pair_double_generator(6, 1, 4) + w.single_generator(6, 0, 5, 1)
    G = ps.PauliSum.jw_fermion(12, terms)
    R = oracle.fermion_sum(12, terms)
    x, z, c = G.export()
    assert _same(x, R.x) and _same(z, R.z) and _same(c, R.c)


@pytest.mark.parametrize("n,kind,n_lo,blocks", [
    (12, 1, 6, [(3, 3)]),
    (16, 1, 8, [(4, 4)]),
    (24, 1, 12, [(6, 6)]),
    (10, 1, 4, [(1, 2)]),
    (12, 1, 6, [(k, 6 - k) for k in range(7)]),
    (14, 1, 7, [(3, 4), (4, 3), (2, 5)]),
    (11, 0, 5, []),
])
def test_sector_rank_unrank_bit_exact(ps, n, kind, n_lo, blocks):
    import torch
    S = ps.Sector(n, kind, n_lo, blocks)
    R = oracle.Sector(n, kind, n_lo, blocks)
    assert S.dim == R.dim
    cfg = R.configs()
    dev = torch.device("cuda")
    idx = S.rank(torch.from_numpy(cfg.astype(np.int64)).to(dev)).cpu().numpy()
    assert _same(idx, np.arange(R.dim, dtype=np.int64))
    back = S.unrank(torch.arange(R.dim, dtype=torch.int64, device=dev)).cpu().numpy().astype(np.uint64)
    assert _same(back, cfg)
    # configurations outside the sector rank to -1; out-of-range indices unrank to all ones
    rng = np.random.default_rng(n)
    probe = rng.integers(0, 1 << n, 4000, dtype=np.uint64)
    gi = S.rank(torch.from_numpy(probe.astype(np.int64)).to(dev)).cpu().numpy()
    assert _same(gi, R.index(probe))
    bad = S.unrank(torch.tensor([-1, R.dim], dtype=torch.int64, device=dev)).cpu().numpy()
    assert np.all(bad == -1)


def test_sector_dims_eq_fcidim(ps):
    for norb, na, nb in [(6, 3, 3), (12, 6, 6), (16, 8, 8), (14, 7, 7), (9, 4, 4)]:
        assert ps.Sector.molecular(norb, na, nb).dim == math.comb(norb, na) * math.comb(norb, nb)
