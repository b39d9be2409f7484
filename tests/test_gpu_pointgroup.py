"""Point-group sectors (pauli_sector_create_irrep) against the oracle: rank and
unrank bit for bit, H psi and <H> on multi-block irrep sectors for every
gather that takes them (staged by pattern, by rank, lists, SVD; one block and
several), rotations, rotation sequences and pool gradients.  Tolerances as
the other GPU tests: 1e-12 (complex128), 1e-5 (complex64) relative."""
import numpy as np
import pytest

import oracle
from oracle import vqe as ovqe
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


def _case(ps, norb, na, nb, gamma, seed=3, single=False):
    irr = w.orbital_irreps(norb, seed=4000 + norb)
    qirr = np.concatenate([irr, irr])
    blocks = w.pointgroup_blocks(norb, na, nb, gamma, irr)
    if single:
        blocks = blocks[-1:]
    h, g = w.pointgroup_integrals(norb, seed, irr)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    S = ps.Sector.irrep_blocks(2 * norb, norb, blocks, qirr)
    So = oracle.Sector.irrep_blocks(2 * norb, norb, blocks, qirr)
    assert S.dim == So.dim and S.dim > 0
    return H, R, S, So, irr, qirr, blocks


@pytest.mark.parametrize("norb,na,nb,gamma", [(6, 3, 3, 0), (7, 2, 4, 5), (12, 3, 3, 6)])
def test_pointgroup_rank_unrank(ps, norb, na, nb, gamma):
    import torch
    H, R, S, So, irr, qirr, blocks = _case(ps, norb, na, nb, gamma)
    cfg = So.configs().astype(np.int64)
    got = S.rank(torch.from_numpy(cfg).cuda()).cpu().numpy()
    assert np.array_equal(got, np.arange(So.dim))
    back = S.unrank(torch.arange(So.dim, device="cuda")).cpu().numpy()
    assert np.array_equal(back, cfg)
    rng = np.random.default_rng(norb)
    probes = rng.integers(0, 1 << (2 * norb), 500)
    ref = So.index(probes.astype(np.uint64))
    assert np.array_equal(S.rank(torch.from_numpy(probes).cuda()).cpu().numpy(), ref)


SHAPES = [(4, 1, 1, 0, 0), (1, 2, 4, 0, 0), (2, 1, 16, 0, 1), (4, 1, 1, 0, 1), (1, 1, 4, 3, 0), (1, 1, 1, 4, 1),
          (2, 1, 1, 4, 1)]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb,gamma,single", [(6, 3, 3, 0, False), (8, 4, 4, 3, False), (7, 2, 4, 5, False),
                                                     (8, 4, 4, 3, True)])
def test_pointgroup_apply_and_expect(ps, dt, norb, na, nb, gamma, single):
    import torch
    H, R, S, So, irr, qirr, blocks = _case(ps, norb, na, nb, gamma, single=single)
    psi = _rounded(w.random_state(S.dim, 60 + norb), dt)
    ref = oracle.apply(So, R, psi)
    E = oracle.expect(So, R, psi)[0]
    x = torch.from_numpy(psi).to("cuda", _tdt(dt))
    out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(out - ref) <= TOL[dt] * np.linalg.norm(ref)
    ps.prepare(H, S)
    for t, nbuf, split, direct, ranked in SHAPES:
        if direct in (3, 4) and len(blocks) != 1:
            continue
        ps.set_launch_config(H, S, _tdt(dt), ps.LaunchConfig(cols_per_thread=t, staged_rows=nbuf, row_split=split,
                                                             direct=direct, ranked=ranked, ms=0.0))
        out = ps.apply(H, S, x).cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(out - ref) <= TOL[dt] * np.linalg.norm(ref), (t, nbuf, split, direct, ranked)
        r = ps.expect(H, S, x).cpu().numpy()
        assert abs(complex(r[0], r[1]) - E) <= (1e-12 if dt == "c128" else 1e-6) * max(1.0, abs(E))


def test_pointgroup_rotations_sequences_and_pool(ps):
    import torch
    norb, na, nb = 6, 3, 3
    for single in (False, True):
        H, R, S, So, irr, qirr, blocks = _case(ps, norb, na, nb, 0, single=single)
        # symmetry-adapted generators: excitations that keep the irrep (equal labels)
        pool = [(lab, t) for lab, t in w.uccsd_pool(norb, na, nb)]
        def keeps(label):
            # labels s{a,b}_p_q (single p -> q) and d.._ij_ab (double ij -> ab), orbitals < 10
            kind, src, dst = label.split("_")
            if kind in ("sa", "sb"):
                return irr[int(src)] == irr[int(dst)]
            i, j, a, b = int(src[0]), int(src[1]), int(dst[0]), int(dst[1])
            return (irr[i] ^ irr[j]) == (irr[a] ^ irr[b])
        pool = [p for p in pool if keeps(p[0])][:40]
        assert len(pool) >= 5
        gens = [ps.PauliSum.jw_fermion(2 * norb, t) for _, t in pool]
        gens_or = [oracle.fermion_sum(2 * norb, t) for _, t in pool]
        psi = w.random_state(S.dim, 5)
        th = np.random.default_rng(1).uniform(-0.5, 0.5, len(gens))
        # one rotation, a sequence of rotations (fused on one block), pool gradients
        x = torch.from_numpy(psi).cuda()
        ps.rotate(gens[0], S, th[0], x)
        ref = oracle.rotate(So, gens_or[0], th[0], psi)
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-12
        y = torch.from_numpy(psi).cuda()
        Q = ps.RotSeq(gens, S)
        Q.apply(th, y)
        ref = psi.copy()
        for G, t in zip(gens_or, th):
            ref = oracle.rotate(So, G, t, ref)
        assert np.linalg.norm(y.cpu().numpy() - ref) <= 1e-12
        for G in gens:
            assert G.status() == 0
        hp = torch.from_numpy(oracle.apply(So, R, psi)).cuda()
        P = ps.Pool(gens, S)
        g = P.gradients(torch.from_numpy(psi).cuda(), hp).cpu().numpy()
        gref = ovqe.pool_gradients(So, R, gens_or, psi)
        assert np.abs(g - gref).max() <= 1e-11 * max(1.0, np.abs(gref).max())


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_pointgroup_batch(ps, dt):
    """Single-block irrep sectors in one batched launch, mixed with a plain
    (popcount) molecular sector: every installed shape (uniform pattern or rank
    staging, per-state groups) gives each state's H psi and <H> of the oracle."""
    import torch
    cases = [_case(ps, 6, 3, 3, 0, seed=s, single=True) for s in (3, 4)] + \
            [_case(ps, 8, 4, 4, 3, seed=5, single=True)]
    h, g = w.molecular_integrals(7, 2)
    Hm = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    Rm = oracle.jw_hamiltonian(7, h, g, eps_drop=1e-12)
    Sm, Smo = ps.Sector.molecular(7, 3, 4), oracle.Sector.molecular(7, 3, 4)
    Hs = [c[0] for c in cases] + [Hm]
    Rs = [c[1] for c in cases] + [Rm]
    Ss = [c[2] for c in cases] + [Sm]
    Sos = [c[3] for c in cases] + [Smo]
    psis = [_rounded(w.random_state(S.dim, 90 + i), dt) for i, S in enumerate(Ss)]
    refs = [oracle.apply(So, R, p) for So, R, p in zip(Sos, Rs, psis)]
    Es = [oracle.expect(So, R, p)[0] for So, R, p in zip(Sos, Rs, psis)]
    xs = [torch.from_numpy(p).to("cuda", _tdt(dt)) for p in psis]
    outs = [torch.empty_like(x) for x in xs]
    B = ps.Batch(Hs, Ss, dtype=_tdt(dt))
    res = torch.empty((len(Ss), 4), dtype=torch.float64, device="cuda")
    for shape in (None, ps.LaunchConfig(cols_per_thread=2, staged_rows=1, row_split=1, direct=0, ranked=0, ms=0.0),
                  ps.LaunchConfig(cols_per_thread=0, staged_rows=1, row_split=1, direct=0, ranked=0, ms=0.0)):
        if shape is not None:
            B.set_launch_config(shape)
        for o in outs:
            o.zero_()
        B.apply(xs, outs, res)
        r = res.cpu().numpy()
        for i in range(len(Ss)):
            got = outs[i].cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(got - refs[i]) <= TOL[dt] * np.linalg.norm(refs[i]), (shape, i)
            assert abs(complex(r[i, 0], r[i, 1]) - Es[i]) <= (1e-12 if dt == "c128" else 1e-6) * max(1.0, abs(Es[i]))
