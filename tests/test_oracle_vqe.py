"""Pins of the variational oracle (oracle/vqe.py): the product-ansatz energy
and its gradient by definition, against finite differences, the variational
bound and closed forms."""
import numpy as np

import oracle
from oracle import dense, vqe
import workloads as w

NORB = 4


def _problem(R=1.3, count=8, seed=5):
    h0, h1, g0 = w.pes_integrals(NORB, w.PES_SEED)
    h, g = w.pes_point(h0, h1, g0, R)
    H = oracle.jw_hamiltonian(NORB, h, g, eps_drop=1e-12)
    s = oracle.Sector.molecular(NORB, 2, 2)
    pairs = w.pair_double_ansatz(NORB, count)
    gens = [oracle.fermion_sum(2 * NORB, w.pair_double_generator(NORB, p, q)) for p, q in pairs]
    ref = int(s.index(oracle.hf_config(NORB, 2, 2))[0])
    theta = np.random.default_rng(seed).uniform(-0.6, 0.6, count)
    return h, g, H, s, gens, ref, theta


def test_gradient_matches_central_differences():
    _, _, H, s, gens, ref, theta = _problem()
    g = vqe.gradient(s, H, gens, theta, ref)
    step = 1e-5
    fd = np.zeros_like(theta)
    for k in range(len(theta)):
        e = np.zeros_like(theta)
        e[k] = step
        fd[k] = (vqe.energy(s, H, gens, theta + e, ref) - vqe.energy(s, H, gens, theta - e, ref)) / (2 * step)
    assert np.abs(g).max() > 1e-2  # a non-trivial point
    assert np.abs(g - fd).max() < 1e-7


def test_energy_obeys_the_variational_bound():
    _, _, H, s, gens, ref, _ = _problem()
    Hs = dense.sector_matrix(2 * NORB, H.x, H.z, H.c, s.configs())
    e0 = np.linalg.eigvalsh(Hs)[0]
    for seed in range(4):
        theta = np.random.default_rng(seed).uniform(-np.pi, np.pi, len(gens))
        psi = vqe.state(s, gens, theta, ref)
        assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
        assert vqe.energy(s, H, gens, theta, ref) >= e0 - 1e-10


def test_zero_angles_give_the_hartree_fock_energy():
    h, g, H, s, gens, ref, _ = _problem()
    e = vqe.energy(s, H, gens, np.zeros(len(gens)), ref)
    assert abs(e - oracle.hf_energy(NORB, h, g, 2, 2)) < 1e-12


def test_pair_double_generator_has_period_two_pi():
    """A pair double G = i(T - T^dagger) has spectrum {-1, 0, 1}: exp(-2 pi i G) = 1,
    and exp(-i pi/2 G) moves the pair completely (|<target|U|ref>| = 1)."""
    _, _, H, s, gens, ref, _ = _problem()
    psi = w.random_state(s.dim, 9)
    assert np.allclose(oracle.rotate(s, gens[0], 2 * np.pi, psi), psi, atol=1e-12)
    e_ref = np.zeros(s.dim, complex)
    e_ref[ref] = 1.0
    # pair (0, 1): orbital 0 doubly occupied in the reference, orbital 1 too;
    # pair (0, 2): moves the 0 pair into the empty orbital 2
    p, q = w.pair_double_ansatz(NORB, 2)[1]
    G = oracle.fermion_sum(2 * NORB, w.pair_double_generator(NORB, p, q))
    out = oracle.rotate(s, G, np.pi / 2, e_ref)
    moved = oracle.hf_config(NORB, 2, 2) & ~((1 << p) | (1 << (NORB + p))) | (1 << q) | (1 << (NORB + q))
    assert abs(abs(out[int(s.index(moved)[0])]) - 1.0) < 1e-12


def test_pool_gradients_match_finite_differences():
    """ADAPT's <psi|[H, A_k]|psi> is the derivative at t = 0 of
    <psi|exp(i t G_k) H exp(-i t G_k)|psi> (A_k = -i G_k)."""
    _, _, H, s, _, ref, _ = _problem()
    pool = w.uccsd_pool(NORB, 2, 2)
    gens = [oracle.fermion_sum(2 * NORB, terms) for _, terms in pool]
    psi = w.random_state(s.dim, 77)
    g = vqe.pool_gradients(s, H, gens, psi)
    step = 1e-5
    for k, G in enumerate(gens):
        ep = oracle.expect(s, H, oracle.rotate(s, G, step, psi))[0].real
        em = oracle.expect(s, H, oracle.rotate(s, G, -step, psi))[0].real
        assert abs(g[k] - (ep - em) / (2 * step)) < 1e-7, k
    assert np.abs(g).max() > 1e-2


def test_pool_gradient_of_a_commuting_generator_is_zero():
    """The total particle-number-like generator sum_p n_p commutes with H: its
    gradient vanishes for any state (pin of a dropped or mis-signed term)."""
    _, _, H, s, _, ref, _ = _problem()
    terms = [(1.0, [(p, 1), (p, 0)]) for p in range(2 * NORB)]
    N = oracle.fermion_sum(2 * NORB, terms)
    psi = w.random_state(s.dim, 78)
    assert abs(vqe.pool_gradients(s, H, [N], psi)[0]) < 1e-12


def test_pair_doubles_keep_the_seniority_zero_configurations():
    """The reading behind the row-restricted energy of the 32-qubit scan: every
    generalized pair double maps the configurations whose beta string equals the
    alpha string onto themselves, so a product of them applied to the closed-shell
    reference vanishes off that set, and <psi|H|psi> over the set equals the full
    expectation (checked with the oracle's own apply)."""
    norb, npair = 6, 3
    s = oracle.Sector.molecular(norb, npair, npair)
    cfg = s.configs()
    sz = set(int(c) for c in w.seniority_zero_configs(norb, npair))
    assert len(sz) == 20 and all(c in set(int(x) for x in cfg) for c in sz)
    mask = np.array([int(c) in sz for c in cfg])
    for p, q in w.pair_double_ansatz(norb, 15):
        G = oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, p, q))
        for idx in np.flatnonzero(mask):
            e = np.zeros(len(cfg), complex)
            e[idx] = 1.0
            out = oracle.apply(s, G, e)
            assert np.abs(out[~mask]).max(initial=0.0) == 0.0, (p, q, int(cfg[idx]))
    # a product state of the ansatz and its energy from the set alone
    h0, h1, g0 = w.pes_integrals(norb, w.PES_SEED)
    h, g = w.pes_point(h0, h1, g0, 1.7)
    H = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    gens = [oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, p, q))
            for p, q in w.pair_double_ansatz(norb, 15)]
    ref = int(s.index(oracle.hf_config(norb, npair, npair))[0])
    theta = np.random.default_rng(3).uniform(-0.5, 0.5, len(gens))
    psi = np.zeros(len(cfg), complex)
    psi[ref] = 1.0
    for G, t in zip(gens, theta):
        psi = oracle.rotate(s, G, t, psi)
    assert np.abs(psi[~mask]).max() == 0.0
    hp = oracle.apply(s, H, psi)
    e_full = np.vdot(psi, hp).real
    e_rows = np.vdot(psi[mask], hp[mask]).real
    assert abs(e_full - e_rows) <= 1e-13 * max(1.0, abs(e_full))
