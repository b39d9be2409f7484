"""Pins of the oracle's Jordan-Wigner build (Sec. 2.3, Algorithm 1) and sectors (Sec. 2.4)."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Jordan-Wigner
# ---------------------------------------------------------------------------
def test_anticommutators_exact():
    """{a_P, a_Q^dagger} = delta_PQ I and {a_P, a_Q} = 0, as canonical Pauli sums, bit-exact."""
    n = 6
    for P in range(n):
        for Q in range(n):
            aP, aQd, aQ = oracle.ladder(n, P, False), oracle.ladder(n, Q, True), oracle.ladder(n, Q, False)
            ac = oracle.sum_add(oracle.sum_product(aP, aQd), oracle.sum_product(aQd, aP))
            if P == Q:
                assert ac.m == 1 and int(ac.x[0]) == 0 and int(ac.z[0]) == 0 and ac.c[0] == 1.0
            else:
                assert ac.m == 0
            aa = oracle.sum_add(oracle.sum_product(aP, aQ), oracle.sum_product(aQ, aP))
            assert aa.m == 0


def test_ladder_matches_occupation_number_definition():
    n = 5
    for P in range(n):
        a = oracle.ladder(n, P, False)
        assert np.array_equal(dense.pauli_sum_matrix(n, a.x, a.z, a.c), dense.annihilator(n, P).toarray())


@pytest.mark.parametrize("norb,seed,e_nn", [(2, 3, 0.0), (3, 4, 0.7), (4, 5, -1.25)])
def test_jw_hamiltonian_matches_fermionic_matrix(norb, seed, e_nn):
    """Pauli sum of Algorithm 1 == H_elec built from ladder matrices (eq. second_quantized_hamiltonian)."""
    h, g = w.molecular_integrals(norb, seed)
    H = oracle.jw_hamiltonian(norb, h, g, e_nn=e_nn)
    Hp = dense.pauli_sum_matrix(2 * norb, H.x, H.z, H.c)
    Hf = dense.fermionic_hamiltonian(norb, h, g, e_nn=e_nn)
    assert np.abs(Hp - Hf).max() <= 1e-13 * max(1.0, np.abs(Hf).max())


def test_jw_raw_entry_count():
    """4 raw entries per one-body integral, 16 per two-body term with P != R and Q != S."""
    norb = 12
    h, g = w.MOL24.integrals()
    x, z, c = oracle.jw_raw(norb, h, g)
    n1 = 2 * norb * norb
    same = norb ** 4 - (2 * norb ** 3 - norb ** 2)  # same spin, p != r and q != s
    n2 = 2 * same + 2 * norb ** 4
    assert len(x) == 4 * n1 + 16 * n2 == 1_222_272


@pytest.mark.parametrize("norb", [6, 8])
def test_hamiltonian_is_hermitian(norb):
    """Every letter-form coefficient c = C i^-#Y of the reduced H is real (exactly)."""
    h, g = w.molecular_integrals(norb, 0)
    H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    ny = np.array([bin(int(a) & int(b)).count("1") for a, b in zip(H.x, H.z)])
    c_letter = H.c * (1j) ** (-ny)
    assert np.abs(c_letter.imag).max() < 1e-15 * np.abs(H.c).max()


def test_hamiltonian_conserves_particle_numbers(mol12):
    """[H, N_alpha] = [H, N_beta] = 0 with N_sigma = sum_p (1 - Z_p)/2, as Pauli-sum products."""
    _, _, H = mol12
    norb = 6
    for sigma in range(2):
        x = np.zeros(norb + 1, np.uint64)
        z = np.array([0] + [1 << (sigma * norb + p) for p in range(norb)], np.uint64)
        c = np.array([norb / 2] + [-0.5] * norb, dtype=np.complex128)
        N = oracle.canonical(12, x, z, c)
        comm = oracle.sum_add(oracle.sum_product(H, N), oracle.sum_product(N, H), b_scale=-1.0)
        assert comm.m == 0 or np.abs(comm.c).max() < 1e-14


@pytest.mark.parametrize("norb,na,nb,seed", [(3, 2, 1, 1), (3, 1, 1, 2), (4, 2, 2, 3), (4, 3, 1, 4)])
def test_hf_closed_form_matches_fermionic_matrix(norb, na, nb, seed):
    h, g = w.molecular_integrals(norb, seed)
    Hf = dense.fermionic_hamiltonian(norb, h, g, sparse=True)
    b = oracle.hf_config(norb, na, nb)
    assert abs(oracle.hf_energy(norb, h, g, na, nb) - Hf[b, b].real) < 1e-12


def test_hf_energy_equals_pauli_expectation_12_qubits(mol12):
    """E_HF closed form == <HF|H|HF> of the 12-qubit Pauli Hamiltonian (sector (3a,3b))."""
    h, g, H = mol12
    s = oracle.Sector.molecular(6, 3, 3)
    psi = np.zeros(s.dim, complex)
    psi[s.index(oracle.hf_config(6, 3, 3))[0]] = 1.0
    E, _ = oracle.expect(s, H, psi)
    assert abs(E - oracle.hf_energy(6, h, g, 3, 3)) < 1e-12


@pytest.mark.parametrize("norb", [6, 8])
def test_phase_matrix_rank_collapse(norb):
    """Sec. 2.4 / Table 1: off-diagonal X-groups have SVD rank R_g <= 2 and the
    diagonal group has R_0 = n_orb + 2 (tolerance sigma > 1e-12 as in Table 1)."""
    h, g = w.molecular_integrals(norb, 0)
    H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    amask = (1 << norb) - 1
    ranks = {}
    for xg in np.unique(H.x):
        sel = H.x == xg
        za = (H.z[sel] & np.uint64(amask)).astype(np.uint64)
        zb = (H.z[sel] >> np.uint64(norb)).astype(np.uint64)
        ua, ia = np.unique(za, return_inverse=True)
        ub, ib = np.unique(zb, return_inverse=True)
        M = np.zeros((len(ua), len(ub)), complex)
        np.add.at(M, (ia, ib), H.c[sel])
        s = np.linalg.svd(M, compute_uv=False)
        ranks[int(xg)] = int((s > 1e-12).sum())
    assert ranks.pop(0) == norb + 2
    assert max(ranks.values()) <= 2
    # the rank-1 groups dominate, as in every row of Table 1
    assert sum(1 for r in ranks.values() if r == 1) > 0.85 * len(ranks)


def test_terms_per_group_band():
    """Table 2 reports M/G between 4.84 and 5.35 for molecular H; the synthetic
    generator lands in the same regime (5-6.5) for 6-12 orbitals."""
    for norb in (6, 8, 10):
        h, g = w.molecular_integrals(norb, 0)
        H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
        mg = H.m / len(np.unique(H.x))
        assert 5.0 < mg < 6.5


# ---------------------------------------------------------------------------
# sectors
# ---------------------------------------------------------------------------
def test_string_counts_match_enumeration():
    for bits in range(0, 11):
        for k in range(0, bits + 1):
            assert oracle.count_strings(bits, k) == sum(1 for v in range(1 << bits) if bin(v).count("1") == k)


def test_table2_det_column():
    """eq. fcidim: Det = C(No, Na) C(No, Nb) reproduces every Det value of Table 2."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_det.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 11
    for name, basis, ne, no, printed in rows:
        ne, no, printed = int(ne), int(no), float(printed)
        det = oracle.count_strings(no, ne // 2) ** 2
        exp = math.floor(math.log10(printed))
        assert round(det / 10 ** exp, 1) == round(printed / 10 ** exp, 1), (name, basis, det)


@pytest.mark.parametrize("norb,na,nb", [(6, 3, 3), (5, 2, 3), (4, 0, 2), (4, 4, 1)])
def test_molecular_sector_enumeration(norb, na, nb):
    s = oracle.Sector.molecular(norb, na, nb)
    cfg = s.configs()
    assert s.dim == len(cfg) == math.comb(norb, na) * math.comb(norb, nb)
    lo = cfg & np.uint64((1 << norb) - 1)
    hi = cfg >> np.uint64(norb)
    assert all(bin(int(v)).count("1") == na for v in lo)
    assert all(bin(int(v)).count("1") == nb for v in hi)
    assert np.all(np.diff(cfg.astype(np.int64)) > 0)  # one block: ascending numeric order
    assert np.array_equal(s.index(cfg), np.arange(s.dim))
    outside = [v for v in range(1 << (2 * norb)) if bin(v & ((1 << norb) - 1)).count("1") != na][:50]
    assert np.all(s.index(np.array(outside, np.uint64)) == -1)


def test_multiblock_sector():
    """Sz = 0 on a 10-site chain split 5|5: blocks (k, 5-k); dim = C(10,5)."""
    blocks = [(k, 5 - k) for k in range(6)]
    s = oracle.Sector(10, oracle.BLOCKS, 5, blocks)
    cfg = s.configs()
    assert s.dim == math.comb(10, 5) == len(set(cfg.tolist()))
    assert all(bin(int(v)).count("1") == 5 for v in cfg)
    off = 0
    for (kl, kh) in blocks:
        d = math.comb(5, kl) * math.comb(5, kh)
        blk = cfg[off:off + d]
        assert np.all(np.diff(blk.astype(np.int64)) > 0)
        assert all(bin(int(v) & 31).count("1") == kl for v in blk)
        off += d
    assert np.array_equal(s.index(cfg), np.arange(s.dim))


def test_full_sector_is_identity():
    s = oracle.Sector.full(9)
    assert s.dim == 512
    assert np.array_equal(s.configs(), np.arange(512, dtype=np.uint64))
    assert np.array_equal(s.index(np.arange(512, dtype=np.uint64)), np.arange(512))


@pytest.mark.parametrize("n,n_lo,blocks", [(30, 15, [(1, 1), (2, 0), (0, 2)]), (32, 16, [(2, 1), (1, 2)]),
                                           (34, 17, [(1, 1)])])
def test_sector_index_by_binary_search_above_28_qubits(n, n_lo, blocks):
    """Above 28 qubits the oracle finds an index by binary search in the block's
    sorted list instead of a lookup table.  Pinned against positions in an
    enumeration written here (blocks in the given order, high string outer,
    low string inner, both ascending), and against -1 for strings outside."""
    from itertools import combinations
    S = oracle.Sector(n, oracle.BLOCKS, n_lo, blocks)
    n_hi = n - n_lo
    expect_cfg = []
    for k_lo, k_hi in blocks:
        los = sorted(sum(1 << b for b in c) for c in combinations(range(n_lo), k_lo))
        his = sorted(sum(1 << b for b in c) for c in combinations(range(n_hi), k_hi))
        expect_cfg += [lo | (hi << n_lo) for hi in his for lo in los]
    assert S.dim == len(expect_cfg)
    cfg = np.array(expect_cfg, dtype=np.uint64)
    assert np.array_equal(S.configs(), cfg)
    assert np.array_equal(S.index(cfg), np.arange(len(cfg)))
    # outside: wrong popcounts in either half, and a bit at or above n
    rng = np.random.default_rng(n)
    inside = set(expect_cfg)
    probes = [0, 1, (1 << n_lo) | 1 | 2 | 4, (1 << n) - 1, 1 << n, (1 << n) | int(cfg[0])]
    probes += [int(b) for b in rng.integers(0, 1 << n, 200, dtype=np.uint64)]
    probes = [p for p in probes if p not in inside]
    assert np.all(S.index(np.array(probes, dtype=np.uint64)) == -1)


def _brute_irrep_sector(n, n_lo, blocks, qirr):
    def irrep(v, first, bits):
        g = 0
        for j in range(bits):
            if (v >> j) & 1:
                g ^= qirr[first + j]
        return g
    n_hi = n - n_lo
    cfg = []
    for kl, il, kh, ih in blocks:
        los = [v for v in range(1 << n_lo) if bin(v).count("1") == kl and irrep(v, 0, n_lo) == il]
        his = [v for v in range(1 << n_hi) if bin(v).count("1") == kh and irrep(v, n_lo, n_hi) == ih]
        cfg += [lo | (hi << n_lo) for hi in his for lo in los]
    return cfg


@pytest.mark.parametrize("norb,na,nb,gamma", [(6, 3, 3, 0), (7, 2, 4, 5), (15, 1, 2, 3)])
def test_pointgroup_sector_enumeration(norb, na, nb, gamma):
    """Point-group blocks (k_lo, irrep_lo, k_hi, irrep_hi): positions against a
    brute-force enumeration written here (above 28 qubits via the binary search),
    -1 outside, and the block dimensions summing to the (N_a, N_b) count split
    by irrep."""
    irr = w.orbital_irreps(norb)
    qirr = np.concatenate([irr, irr])
    blocks = w.pointgroup_blocks(norb, na, nb, gamma, irr)
    S = oracle.Sector.irrep_blocks(2 * norb, norb, blocks, qirr)
    cfg = _brute_irrep_sector(2 * norb, norb, blocks, qirr)
    assert S.dim == len(cfg)
    assert np.array_equal(S.configs(), np.array(cfg, dtype=np.uint64))
    assert np.array_equal(S.index(np.array(cfg, dtype=np.uint64)), np.arange(len(cfg)))
    # the sectors of all 8 total irreps partition the (N_a, N_b) block
    tot = 0
    for gg in range(8):
        tot += oracle.Sector.irrep_blocks(2 * norb, norb, w.pointgroup_blocks(norb, na, nb, gg, irr), qirr).dim
    assert tot == oracle.Sector.molecular(norb, na, nb).dim
    inside = set(cfg)
    rng = np.random.default_rng(norb)
    probes = [int(v) for v in rng.integers(0, 1 << (2 * norb), 300, dtype=np.uint64) if int(v) not in inside]
    assert np.all(S.index(np.array(probes, dtype=np.uint64)) == -1)


@pytest.mark.parametrize("norb,na,nb", [(5, 2, 2), (6, 3, 2)])
def test_pointgroup_hamiltonian_keeps_its_sectors(norb, na, nb):
    """With integrals that respect the point group, H maps each irrep sector into
    itself: the full-space apply of a state supported on one sector has no weight
    outside it, and equals the oracle's sector apply there (dense check)."""
    irr = w.orbital_irreps(norb, seed=4001)
    qirr = np.concatenate([irr, irr])
    h, g = w.pointgroup_integrals(norb, 3, irr)
    H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    full = oracle.Sector.full(2 * norb)
    for gamma in range(8):
        blocks = w.pointgroup_blocks(norb, na, nb, gamma, irr)
        if not blocks:
            continue
        S = oracle.Sector.irrep_blocks(2 * norb, norb, blocks, qirr)
        cfg = S.configs()
        psi = w.random_state(S.dim, 7 + gamma)
        big = np.zeros(1 << (2 * norb), np.complex128)
        big[cfg.astype(np.int64)] = psi
        out_full = oracle.apply(full, H, big)
        mask = np.ones(1 << (2 * norb), bool)
        mask[cfg.astype(np.int64)] = False
        assert np.abs(out_full[mask]).max() < 1e-12
        assert np.allclose(out_full[cfg.astype(np.int64)], oracle.apply(S, H, psi), atol=1e-12, rtol=0)
