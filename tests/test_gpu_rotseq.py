"""Products of rotations applied tile by tile (pauli_rotseq_*) against the
oracle's rotations applied one after the other, and against pauli_rotate_seq.

Tolerances: ||psi_gpu - psi_oracle|| <= 1e-12 (complex128) and 1e-5
(complex64) for the unit-norm states here, the oracle run on the
complex64-rounded input."""
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


def _oracle_seq(So, gens_or, thetas, psi):
    v = psi.copy()
    for G, t in zip(gens_or, thetas):
        v = oracle.rotate(So, G, float(t), v)
    return v


def _run(ps, norb, na, nb, order, dt, seed, extra_diag=True):
    import torch
    pool = w.uccsd_pool(norb, na, nb)
    if order == "trotter":
        pool = w.uccsd_trotter_order(pool, norb)
    elif order == "shuffled":
        idx = np.random.default_rng(seed).permutation(len(pool))
        pool = [pool[i] for i in idx]
    terms = [t for _, t in pool]
    if extra_diag:
        # diagonal generators (number operators) placed inside the sequence
        rng = np.random.default_rng(seed + 1)
        for pos in sorted(rng.choice(len(terms), 3, replace=False), reverse=True):
            wts = rng.normal(size=2 * norb)
            terms.insert(int(pos), [(float(wts[p]), [(p, 1), (p, 0)]) for p in range(2 * norb)])
    gens_dev = [ps.PauliSum.jw_fermion(2 * norb, t) for t in terms]
    gens_or = [oracle.fermion_sum(2 * norb, t) for t in terms]
    S = ps.Sector.molecular(norb, na, nb)
    So = oracle.Sector.molecular(norb, na, nb)
    thetas = np.random.default_rng(seed).uniform(-0.4, 0.4, len(terms))
    psi = w.random_state(S.dim, seed)
    if dt == "c64":
        psi = psi.astype(np.complex64).astype(np.complex128)
    Q = ps.RotSeq(gens_dev, S)
    x = torch.from_numpy(psi).to("cuda", _tdt(dt))
    Q.apply(thetas, x)
    out = x.cpu().numpy().astype(np.complex128)
    ref = _oracle_seq(So, gens_or, thetas, psi)
    for G in gens_dev:
        assert G.status() == 0
    return Q, out, ref, gens_dev, S, thetas, psi


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb,order", [(6, 3, 3, "trotter"), (6, 3, 3, "pool"), (6, 2, 3, "shuffled"),
                                              (8, 4, 4, "trotter"), (7, 3, 2, "shuffled")])
def test_rotseq_matches_sequential_oracle(ps, dt, norb, na, nb, order):
    Q, out, ref, gens, S, thetas, psi = _run(ps, norb, na, nb, order, dt, 10 + norb)
    assert np.linalg.norm(out - ref) <= TOL[dt] * max(1.0, np.linalg.norm(ref))
    info = Q.info(_tdt(dt))
    assert info["fused"] == len(gens)  # every generator ran inside a fused tile
    if order == "trotter":
        # alpha run, beta run, one run per beta excitation of the alpha-beta doubles
        n_beta_exc = nb * (norb - nb)
        assert info["launches"] == 2 + n_beta_exc, info


def test_rotseq_fused_equals_rotate_seq_24_qubits(ps):
    """The Trotterised UCCSD step of the 24-qubit molecule (1,818 generators,
    38 launches) against 1,818 pauli_rotate launches on the GPU, both precisions."""
    import torch
    norb, na, nb = 12, 6, 6
    pool = w.uccsd_trotter_order(w.uccsd_pool(norb, na, nb), norb)
    gens = [ps.PauliSum.jw_fermion(2 * norb, t) for _, t in pool]
    S = ps.Sector.molecular(norb, na, nb)
    thetas = np.random.default_rng(24).uniform(-0.3, 0.3, len(gens))
    Q = ps.RotSeq(gens, S)
    assert Q.info(torch.complex64) == {"launches": 38, "fused": 1818}
    psi = w.random_state(S.dim, 24)
    for dt in ("c128", "c64"):
        a = torch.from_numpy(psi).to("cuda", _tdt(dt))
        b = a.clone()
        Q.apply(thetas, a)
        ps.rotate_seq(gens, S, thetas, b)
        d = np.linalg.norm((a - b).cpu().numpy().astype(np.complex128))
        assert d <= TOL[dt] * 3, (dt, d)
        assert abs(torch.linalg.vector_norm(a.to(torch.complex128)).item() - 1.0) <= (1e-12 if dt == "c128" else 1e-5)


@pytest.mark.parametrize("kind", ["full", "sz0"])
def test_rotseq_other_sectors_fall_back(ps, kind):
    """Full space and several blocks take one pauli_rotate per generator."""
    import torch
    n = 10
    gens_t = []
    for i in range(n - 1):
        xm = (1 << i) | (1 << (i + 1))
        gens_t.append(([xm, xm], [0, xm], [0.5, 0.5]))  # XX + YY bond
    gens_t.append(([0, 0], [1, 6], [0.3, -0.2]))
    if kind == "full":
        S, So = ps.Sector.full(n), oracle.Sector.full(n)
    else:
        blocks = [(k, 5 - k) for k in range(6)]
        S, So = ps.Sector(n, ps.BLOCKS, 5, blocks), oracle.Sector(n, oracle.BLOCKS, 5, blocks)
    gd = [ps.PauliSum.from_terms(n, a, b, c) for a, b, c in gens_t]
    go = [oracle.build_sum(n, np.array(a, np.uint64), np.array(b, np.uint64), None, np.array(c), np.zeros(len(c)))
          for a, b, c in gens_t]
    th = np.linspace(-0.5, 0.7, len(gd))
    psi = w.random_state(So.dim, 3)
    Q = ps.RotSeq(gd, S)
    assert Q.info(torch.complex128) == {"launches": len(gd), "fused": 0}
    x = torch.from_numpy(psi).to("cuda")
    Q.apply(th, x)
    ref = _oracle_seq(So, go, th, psi)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-12


def test_rotseq_leak_sets_the_generator_status(ps):
    """A single string that changes the alpha particle number inside a fused
    run: its status word reports PAULI_ESECTOR, like pauli_rotate."""
    import torch
    norb = 6
    S = ps.Sector.molecular(norb, 3, 3)
    good = ps.PauliSum.jw_fermion(2 * norb, w.single_generator(norb, 0, 4, 0))
    bad = ps.PauliSum.from_terms(2 * norb, [1 << 2], [0], [1.0])  # X on alpha orbital 2
    Q = ps.RotSeq([good, bad, good], S)
    x = torch.from_numpy(w.random_state(S.dim, 1)).to("cuda")
    Q.apply([0.1, 0.2, 0.3], x)
    assert bad.status() == ps.ESECTOR
    assert good.status() == 0
