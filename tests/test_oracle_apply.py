"""Pins of the oracle's operator-state products against dense Kronecker-built matrices
and against closed-form free-fermion spectra of lattice chains."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle import dense
import workloads as w


def _restrict(Hs, cfg):
    idx = cfg.astype(np.int64)
    return Hs[idx][:, idx]


def test_apply_matches_dense_12_qubits(mol12, mol12_dense):
    """(3a,3b) sector of the 12-qubit molecule: source-form apply == dense 4096x4096 H restricted."""
    _, _, H = mol12
    s = oracle.Sector.molecular(6, 3, 3)
    psi = w.random_state(s.dim, w.MOL12.psi_seed)
    ref = _restrict(mol12_dense, s.configs()) @ psi
    out = oracle.apply(s, H, psi)
    assert np.linalg.norm(out - ref) <= 1e-13 * np.linalg.norm(ref)
    # the full 2^12 space too
    full = oracle.Sector.full(12)
    psi_f = w.random_state(4096, 5)
    out_f = oracle.apply(full, H, psi_f)
    ref_f = mol12_dense @ psi_f
    assert np.linalg.norm(out_f - ref_f) <= 1e-13 * np.linalg.norm(ref_f)


@pytest.mark.parametrize("seed", [0, 1])
def test_apply_general_complex_sum_full_space(seed):
    """Non-Hermitian complex Pauli sum (letter form with phases) on 8 qubits."""
    n = 8
    x, z, gamma, cre, cim = w.random_pauli_terms(n, 60, seed)
    S = oracle.build_sum(n, x, z, gamma, cre, cim)
    Hd = dense.pauli_sum_matrix(n, S.x, S.z, S.c)
    full = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 40 + seed)
    assert np.allclose(oracle.apply(full, S, psi), Hd @ psi, rtol=0, atol=1e-13)


def test_apply_multiblock_sector_xxz():
    """Open XXZ chain, 10 sites, Sz = 0 as blocks (k, 5-k) over the split 5|5."""
    n = 10
    x, z, cre, cim = w.xxz_terms(n, 1)
    S = oracle.build_sum(n, x, z, None, cre, cim)
    Hd = dense.pauli_sum_matrix(n, S.x, S.z, S.c, sparse=True)
    s = oracle.Sector(n, oracle.BLOCKS, 5, [(k, 5 - k) for k in range(6)])
    psi = w.random_state(s.dim, 3)
    ref = _restrict(Hd, s.configs()) @ psi
    assert np.allclose(oracle.apply(s, S, psi), ref, rtol=0, atol=1e-13)
    # H conserves Sz: the sector block of H equals H on the embedded vector
    emb = np.zeros(1 << n, complex)
    emb[s.configs().astype(np.int64)] = psi
    assert np.allclose((Hd @ emb)[s.configs().astype(np.int64)], ref, atol=1e-13)


def test_apply_rows_equals_apply(mol12):
    _, _, H = mol12
    s = oracle.Sector.molecular(6, 3, 3)
    psi = w.random_state(s.dim, 4)
    out = oracle.apply(s, H, psi)
    rows = np.array([0, 1, 7, 199, 200, 398, 399])
    assert np.allclose(oracle.apply_rows(s, H, psi, rows), out[rows], rtol=0, atol=1e-13)


def test_expect_and_hermiticity(mol12, mol12_dense):
    _, _, H = mol12
    s = oracle.Sector.molecular(6, 3, 3)
    Hr = _restrict(mol12_dense, s.configs())
    psi = w.random_state(s.dim, 6)
    phi = w.random_state(s.dim, 7)
    E, n2 = oracle.expect(s, H, psi)
    assert abs(E - np.vdot(psi, Hr @ psi)) < 1e-12
    assert abs(E.imag) < 1e-14
    assert abs(n2 - np.linalg.norm(Hr @ psi) ** 2) < 1e-11
    lhs = np.vdot(phi, oracle.apply(s, H, psi))
    rhs = np.conj(np.vdot(psi, oracle.apply(s, H, phi)))
    assert abs(lhs - rhs) < 1e-12


def test_rotate_single_string_closed_form():
    """exp(-i theta P) = cos(theta) I - i sin(theta) P for a Pauli string P (P^2 = I)."""
    n = 6
    # letter string X0 Y2 Z3 with real coefficient 1 (Hermitian)
    P = oracle.build_sum(n, np.array([0b101], np.uint64), np.array([0b1100], np.uint64), None,
                         np.array([1.0]), np.array([0.0]))
    full = oracle.Sector.full(n)
    psi = w.random_state(1 << n, 8)
    Pd = dense.pauli_sum_matrix(n, P.x, P.z, P.c)
    for theta in (0.3, -1.1, math.pi / 2):
        out = oracle.rotate(full, P, theta, psi)
        ref = math.cos(theta) * psi - 1j * math.sin(theta) * (Pd @ psi)
        assert np.allclose(out, ref, rtol=0, atol=1e-14)
    assert np.allclose(oracle.rotate(full, P, math.pi / 2, psi), -1j * (Pd @ psi), atol=1e-14)


def test_rotate_group_matches_expm():
    """One X-group of a molecular H (8 qubits) and a pair-double generator vs scipy expm."""
    norb = 4
    h, g = w.molecular_integrals(norb, 11)
    H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    s = oracle.Sector.molecular(norb, 2, 2)
    cfg = s.configs().astype(np.int64)
    xs, counts = np.unique(H.x, return_counts=True)
    gx = xs[np.argmax(counts * (xs != 0))]
    sel = H.x == gx
    G = oracle.PauliSum(2 * norb, H.x[sel], H.z[sel], H.c[sel])
    Gp = oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, 0, 2))
    for Gs in (G, Gp):
        assert not oracle.leaks(s, Gs)
        Gd = dense.pauli_sum_matrix(2 * norb, Gs.x, Gs.z, Gs.c)
        assert np.allclose(Gd, Gd.conj().T)
        psi = w.random_state(s.dim, 9)
        for theta in (0.37, -2.2):
            U = sla.expm(-1j * theta * Gd)[np.ix_(cfg, cfg)]
            assert np.allclose(oracle.rotate(s, Gs, theta, psi), U @ psi, rtol=0, atol=1e-13)


def test_pair_double_on_hf_is_a_givens_rotation():
    """exp(theta tau)|HF> = cos(theta)|HF> +- sin(theta)|D> for a pair double p -> q."""
    norb, na = 4, 2
    s = oracle.Sector.molecular(norb, na, na)
    G = oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, 1, 3))
    hf = oracle.hf_config(norb, na, na)
    d = hf ^ ((1 << 1) | (1 << 3)) ^ (((1 << 1) | (1 << 3)) << norb)
    psi = np.zeros(s.dim, complex)
    psi[s.index(hf)[0]] = 1.0
    theta = 0.61
    out = oracle.rotate(s, G, theta, psi)
    i_hf, i_d = s.index(hf)[0], s.index(d)[0]
    assert abs(out[i_hf] - math.cos(theta)) < 1e-14
    assert abs(abs(out[i_d]) - math.sin(theta)) < 1e-14 and abs(out[i_d].imag) < 1e-14
    rest = np.delete(out, [i_hf, i_d])
    assert np.abs(rest).max() < 1e-15


def test_leak_detection():
    """A single JW string of a pair double leaks out of the (Na, Nb) sector; the whole group does not."""
    norb = 4
    s = oracle.Sector.molecular(norb, 2, 2)
    G = oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, 0, 2))
    assert not oracle.leaks(s, G)
    one = oracle.PauliSum(G.n, G.x[:1], G.z[:1], G.c[:1])
    assert oracle.leaks(s, one)


def test_rotate_is_unitary_and_additive(mol12):
    _, _, H = mol12
    s = oracle.Sector.molecular(6, 3, 3)
    xs = np.unique(H.x)
    sel = H.x == xs[len(xs) // 2]
    G = oracle.PauliSum(12, H.x[sel], H.z[sel], H.c[sel])
    psi = w.random_state(s.dim, 10)
    a = oracle.rotate(s, G, 0.4, oracle.rotate(s, G, 0.3, psi))
    b = oracle.rotate(s, G, 0.7, psi)
    assert np.allclose(a, b, atol=1e-13)
    assert abs(np.linalg.norm(b) - 1.0) < 1e-13


def _merge_low_masks(R, n_lo):
    """Rewrite every term X^x Z^z with popc(x_lo) even as the term on the smaller
    of z_lo and z_lo ^ x_lo, its coefficient times (-1)^(popc(x_lo)/2) when the
    mask changed (the segment merge of single-block sectors)."""
    lo = (1 << n_lo) - 1
    zs, cs = [], []
    for xv, zv, cv in zip(R.x.tolist(), R.z.tolist(), R.c.tolist()):
        xl, zl = xv & lo, zv & lo
        p = bin(xl).count("1")
        if p % 2 == 0 and (zl ^ xl) < zl:
            zv ^= xl
            cv = cv * (-1) ** (p // 2)
        zs.append(zv)
        cs.append(cv)
    return oracle.canonical(R.n, R.x.copy(), np.array(zs, np.uint64), np.array(cs, np.complex128))


@pytest.mark.parametrize("norb,na,nb", [(4, 2, 2), (5, 2, 3), (5, 1, 1)])
def test_low_mask_merge_is_exact_on_single_block_sectors(norb, na, nb):
    """On a single-block sector a target t and its source t ^ x share the
    low-half popcount, so half of the bits of x_lo are set in the source and
    z_lo ^ x_lo carries the phase of z_lo times (-1)^(popc(x_lo)/2): the merged
    operator has the same sector projection.  On the full space it differs."""
    h, g = w.molecular_integrals(norb, 4)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    Rm = _merge_low_masks(R, norb)
    assert Rm.m < R.m
    So = oracle.Sector.molecular(norb, na, nb)
    psi = w.random_state(So.dim, 8)
    a, b = oracle.apply(So, R, psi), oracle.apply(So, Rm, psi)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)
    Sf = oracle.Sector.full(2 * norb)
    phi = w.random_state(Sf.dim, 9)
    assert np.linalg.norm(oracle.apply(Sf, R, phi) - oracle.apply(Sf, Rm, phi)) > 1e-3


def test_low_mask_merge_needs_a_single_block():
    """With blocks of different low popcount an X mask with two low bits can move
    a target of block (1, 3) to a source in block (3, 1), where half of x_lo is
    not set in the source: the merged operator differs on that sector."""
    n, n_lo = 8, 4
    rng = np.random.default_rng(2)
    xm = 0b00110011
    zs = [0, 0b1, 0b10, 0b11, 0b10000, 0b100001]
    R = oracle.build_sum(n, np.full(len(zs), xm, np.uint64), np.array(zs, np.uint64), None,
                         rng.normal(size=len(zs)), rng.normal(size=len(zs)), letter_form=False)
    So = oracle.Sector(n, oracle.BLOCKS, n_lo, [(1, 3), (3, 1), (2, 2)])
    psi = w.random_state(So.dim, 3)
    Rm = _merge_low_masks(R, n_lo)
    assert Rm.m < R.m
    assert np.linalg.norm(oracle.apply(So, R, psi) - oracle.apply(So, Rm, psi)) > 1e-3
    # restricted to the single block (2, 2) the two agree
    S1 = oracle.Sector(n, oracle.BLOCKS, n_lo, [(2, 2)])
    phi = w.random_state(S1.dim, 4)
    a, b = oracle.apply(S1, R, phi), oracle.apply(S1, Rm, phi)
    assert np.linalg.norm(a - b) <= 1e-13 * max(np.linalg.norm(a), 1.0)


# ----------------------------------------------------------------------------
# lattice models with a free-fermion (Jordan-Wigner) solution: closed-form
# spectra that owe nothing to Kronecker products or to the oracle
# ----------------------------------------------------------------------------
def _dense_from_apply(So, R):
    D = So.dim
    M = np.zeros((D, D), complex)
    for j in range(D):
        e = np.zeros(D, complex)
        e[j] = 1.0
        M[:, j] = oracle.apply(So, R, e)
    return M


def test_transverse_field_ising_spectrum_is_free_fermion():
    """Open transverse-field Ising chain of eq. TFIM with site-dependent couplings,
    H = sum_i J_i Z_i Z_i+1 + sum_i h_i X_i.  A Jordan-Wigner transformation makes
    it quadratic in fermions: its 2^n eigenvalues are sum_k +-L_k over all sign
    choices, with L_k the singular values of the bidiagonal matrix of h (diagonal)
    and J (superdiagonal) (Lieb, Schultz and Mattis 1961; Pfeuty 1970)."""
    import itertools
    n = 8
    rng = np.random.default_rng(21)
    J, h = rng.normal(size=n - 1), rng.normal(size=n)
    xs, zs, cs = [], [], []
    for i in range(n - 1):
        xs.append(0); zs.append((1 << i) | (1 << (i + 1))); cs.append(J[i])
    for i in range(n):
        xs.append(1 << i); zs.append(0); cs.append(h[i])
    c = np.array(cs)
    R = oracle.build_sum(n, np.array(xs, np.uint64), np.array(zs, np.uint64), None, c, np.zeros_like(c))
    M = _dense_from_apply(oracle.Sector.full(n), R)
    assert np.abs(M - M.conj().T).max() == 0.0
    L = np.linalg.svd(np.diag(h) + np.diag(J, 1), compute_uv=False)
    spec = np.sort([np.dot(sg, L) for sg in itertools.product((-1.0, 1.0), repeat=n)])
    assert np.abs(np.sort(np.linalg.eigvalsh(M)) - spec).max() <= 1e-12 * np.abs(L).sum()


def test_xx_chain_spectra_per_particle_number_are_free_fermion():
    """Open XX chain with fields, H = sum_i J_i (X_i X_i+1 + Y_i Y_i+1) + sum_i h_i Z_i,
    restricted to each fixed-N sector of blocks (k, N - k) over a 5|5 split.  With
    n_i the bit of qubit i, Z_i = 1 - 2 n_i and the bond term hops a particle with
    amplitude 2 J_i, so the N-particle eigenvalues are sum_i h_i plus every sum of N
    eigenvalues of the tridiagonal matrix (-2 h_i on the diagonal, 2 J_i beside it)."""
    import itertools
    n, n_lo = 10, 5
    rng = np.random.default_rng(22)
    J, h = rng.normal(size=n - 1), rng.normal(size=n)
    xs, zs, cs = [], [], []
    for i in range(n - 1):
        b = (1 << i) | (1 << (i + 1))
        xs += [b, b]; zs += [0, b]; cs += [J[i], J[i]]   # X X, Y Y (letter form)
    for i in range(n):
        xs.append(0); zs.append(1 << i); cs.append(h[i])
    c = np.array(cs)
    R = oracle.build_sum(n, np.array(xs, np.uint64), np.array(zs, np.uint64), None, c, np.zeros_like(c))
    eps = np.linalg.eigvalsh(np.diag(-2.0 * h) + np.diag(2.0 * J, 1) + np.diag(2.0 * J, -1))
    for N in range(n + 1):
        blocks = [(k, N - k) for k in range(N + 1) if k <= n_lo and N - k <= n - n_lo]
        So = oracle.Sector(n, oracle.BLOCKS, n_lo, blocks)
        assert So.dim == math.comb(n, N)
        M = _dense_from_apply(So, R)
        spec = np.sort([h.sum() + eps[list(S)].sum() for S in itertools.combinations(range(n), N)])
        assert np.abs(np.sort(np.linalg.eigvalsh(M)) - spec).max() <= 1e-12 * (np.abs(eps).sum() + np.abs(h).sum()), N
