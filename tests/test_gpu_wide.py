"""Multi-word masks (pauli_wsum_*, up to 256 qubits) against the wide oracle,
bit for bit, and against the 64-bit path where both apply.  The 252-qubit
case (126 spatial orbitals, the size of the paper's largest Jordan-Wigner
build) uses a banded synthetic molecule whose identity coefficient also has a
closed form: Tr(H) / 2^n."""
import numpy as np
import pytest

import oracle
from oracle import wide
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _same(dev, ref):
    x, z, c = dev.export()
    assert len(x) == len(ref)
    for i, (xr, zr, cr) in enumerate(ref):
        assert x[i] == xr and z[i] == zr, i
        assert c[i].real == cr.real and c[i].imag == cr.imag, i


def _monomials(n, k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        nf = int(rng.integers(1, 5))
        f = [(int(rng.integers(0, n)), int(rng.integers(0, 2))) for _ in range(nf)]
        out.append((complex(rng.normal(), rng.normal()), f))
    return out


@pytest.mark.parametrize("n,seed", [(72, 1), (130, 2), (256, 3)])
def test_wide_fermion_sums_match_the_oracle(ps, n, seed):
    terms = _monomials(n, 80, seed)
    _same(ps.WidePauliSum.jw_fermion(n, terms), wide.fermion_sum(n, terms))


def test_wide_product_matches_the_oracle(ps):
    n = 100
    ta, tb = _monomials(n, 25, 7), _monomials(n, 20, 8)
    A, B = ps.WidePauliSum.jw_fermion(n, ta), ps.WidePauliSum.jw_fermion(n, tb)
    _same(A @ B, wide.product(n, wide.fermion_sum(n, ta), wide.fermion_sum(n, tb)))


@pytest.mark.parametrize("norb,seed,e_nn", [(6, 0, 0.7), (20, 5, 0.0)])
def test_wide_molecular_equals_the_64_bit_build(ps, norb, seed, e_nn):
    h, g = w.molecular_integrals(norb, seed)
    Wd = ps.WidePauliSum.jw_molecular(h, g, e_nn=e_nn, eps_int=1e-14, eps_drop=1e-12)
    N = ps.PauliSum.jw_molecular(h, g, e_nn=e_nn, eps_int=1e-14, eps_drop=1e-12)
    x, z, c = N.export()
    ref = [(int(a), int(b), complex(cc)) for a, b, cc in zip(x, z, c)]
    _same(Wd, ref)
    gs = Wd.groups()
    _, gs_n = N.groups()
    assert np.array_equal(gs, gs_n)


def _banded_molecule(norb, seed):
    """Tridiagonal h and density-density (pp|rr) for |p - r| <= 1, as monomials
    in the raw order of Algorithm 1 (one-body s, p, q; two-body s, t, p, q, r, u)."""
    rng = np.random.default_rng(seed)
    h = {}
    for p in range(norb):
        h[(p, p)] = rng.normal()
        if p + 1 < norb:
            h[(p, p + 1)] = h[(p + 1, p)] = 0.5 * rng.normal()
    gv = {}
    for p in range(norb):
        for r in range(max(0, p - 1), min(norb, p + 2)):
            if (r, p) in gv:
                gv[(p, r)] = gv[(r, p)]
            else:
                gv[(p, r)] = 0.1 * rng.normal()
    terms = []
    for s in range(2):
        for p in range(norb):
            for q in range(norb):
                if (p, q) in h:
                    terms.append((h[(p, q)], [(s * norb + p, 1), (s * norb + q, 0)]))
    for s in range(2):
        for t in range(2):
            for p in range(norb):
                for r in range(norb):
                    if (p, r) not in gv:
                        continue
                    P, R = s * norb + p, t * norb + r
                    if P == R:
                        continue
                    terms.append((0.5 * gv[(p, r)], [(P, 1), (R, 1), (R, 0), (P, 0)]))
    # Tr(H) / 2^n: n_P has trace 1/2, n_P n_R (P != R) 1/4
    c_id = sum(0.5 * h[(p, p)] for s in range(2) for p in range(norb))
    c_id += sum(0.5 * gv[(p, r)] * 0.25 for s in range(2) for t in range(2) for (p, r) in gv
                if s * norb + p != t * norb + r)
    return terms, c_id


def test_252_qubit_banded_molecule(ps):
    norb = 126
    terms, c_id = _banded_molecule(norb, 11)
    Wd = ps.WidePauliSum.jw_fermion(2 * norb, terms)
    ref = wide.fermion_sum(2 * norb, terms)
    _same(Wd, ref)
    x, z, c = Wd.export()
    assert x[0] == 0 and z[0] == 0  # the identity sorts first
    assert abs(c[0] - c_id) <= 1e-12 * max(1.0, abs(c_id))
    assert max(max(x), max(z)) < (1 << 252)
