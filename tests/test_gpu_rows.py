"""Selected rows of H psi (pauli_expect_rows) against the oracle: the rows'
values element by element (1e-12 complex128, 1e-5 complex64, oracle on the
rounded input), every other entry of the output left as it was, the four
row sums, an index outside the sector (skipped, status PAULI_EINVAL), and a
state that lives on the seniority-zero rows, where the rows give
<psi|H|psi> of the full apply and the same energy gradient of the pair-double
ansatz."""
import numpy as np
import pytest

import oracle
import workloads as w
from test_gpu_parity_shapes import oracle_rows

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


def _cases(ps):
    h, g = w.molecular_integrals(8, 3)
    yield ("mol8", ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12), oracle.jw_hamiltonian(8, h, g, eps_drop=1e-12),
           ps.Sector.molecular(8, 4, 4), oracle.Sector.molecular(8, 4, 4))
    x, z, cre, cim = w.xxz_terms(11, 1)
    yield ("xxz11_full", ps.PauliSum.from_terms(11, x, z, cre, cim),
           oracle.build_sum(11, x, z, np.zeros(len(x), np.uint8), cre, cim),
           ps.Sector.full(11, 5), oracle.Sector.full(11))
    xr, zr, gam, re, im = w.random_pauli_terms(10, 300, 5)
    yield ("random10_blocks", ps.PauliSum.from_terms(10, xr, zr, re, im, gamma=gam),
           oracle.build_sum(10, xr, zr, gam, re, im),
           ps.Sector(10, ps.BLOCKS, 5, [(2, 3), (3, 2), (1, 1)]),
           oracle.Sector(10, oracle.BLOCKS, 5, [(2, 3), (3, 2), (1, 1)]))


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_rows_match_oracle_and_leave_other_entries(ps, dt):
    import torch
    for name, H, R, S, So in _cases(ps):
        rng = np.random.default_rng(len(name))
        rows = np.unique(np.concatenate([rng.choice(S.dim, min(S.dim, 300), replace=False), [0, S.dim - 1]]))
        psi = _rounded(w.random_state(S.dim, 11), dt)
        ref = oracle_rows(So, R, psi, rows)
        x = torch.from_numpy(psi).to("cuda", _tdt(dt))
        out = torch.full_like(x, complex(np.nan, np.nan))
        idx = torch.from_numpy(rows.astype(np.int64)).cuda()
        res = ps.expect_rows(H, S, x, idx, hpsi_out=out).cpu().numpy()
        o = out.cpu().numpy().astype(np.complex128)
        got = o[rows]
        assert np.linalg.norm(got - ref) <= TOL[dt] * np.linalg.norm(ref), name
        mask = np.ones(S.dim, bool)
        mask[rows] = False
        assert np.isnan(o[mask].real).all(), name   # untouched
        # the four sums over the rows (from the stored values)
        p = psi[rows]
        e = np.sum(np.conj(p) * got)
        assert abs(complex(res[0], res[1]) - e) <= 1e-12 * max(1.0, np.abs(p).sum() * np.abs(got).max()), name
        assert abs(res[2] - np.sum(np.abs(got) ** 2)) <= 1e-10 * max(1.0, res[2]), name
        assert abs(res[3] - np.sum(np.abs(p) ** 2)) <= 1e-12, name
        assert H.status() == ps.OK


def test_rows_outside_the_sector_are_skipped(ps):
    import torch
    h, g = w.molecular_integrals(6, 0)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(6, 3, 3)
    psi = torch.from_numpy(w.random_state(S.dim, 2)).cuda()
    out = torch.zeros_like(psi)
    idx = torch.tensor([3, S.dim, -1, 7], dtype=torch.int64, device="cuda")
    res = ps.expect_rows(H, S, psi, idx, hpsi_out=out).cpu().numpy()
    assert H.status() == ps.EINVAL
    good = ps.expect_rows(H, S, psi, torch.tensor([3, 7], dtype=torch.int64, device="cuda")).cpu().numpy()
    assert np.array_equal(res, good)
    assert H.status() == ps.OK
    o = out.cpu().numpy()
    assert np.count_nonzero(o) == 2 and o[3] != 0 and o[7] != 0


def test_seniority_zero_state_energy_and_gradient(ps):
    """A pair-double ansatz state lives on the seniority-zero rows: the rows give
    the full apply's <psi|H|psi> and the same gradient."""
    import torch
    from paper_2606_28952_gb300.pes_scan import make_scan_problem
    norb = 6
    S, ans, make_full, _ = make_scan_problem(norb, 24, torch.complex128, 2, support=False)
    _, _, make_rows, rows = make_scan_problem(norb, 24, torch.complex128, 2, support=True)
    assert rows.numel() == 20
    th = np.random.default_rng(0).uniform(-0.4, 0.4, 24)
    for R in (0.7, 2.2):
        ef, gf = make_full(R)(th)
        er, gr = make_rows(R)(th)
        assert abs(ef - er) <= 1e-12 * max(1.0, abs(ef))
        assert np.abs(gf - gr).max() <= 1e-11 * max(1.0, np.abs(gf).max())
        # and against the oracle's energy of the same state
        eg = make_full(R)
        psi = eg.state(th).cpu().numpy()
        h0, h1, g0 = w.pes_integrals(norb, 2)
        h, g = w.pes_point(h0, h1, g0, R)
        Ro = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
        So = oracle.Sector.molecular(norb, norb // 2, norb // 2)
        assert abs(oracle.expect(So, Ro, psi)[0] - er) <= 1e-11
        # psi really vanishes off the rows
        off = np.ones(S.dim, bool)
        off[rows.cpu().numpy()] = False
        assert np.abs(psi[off]).max() == 0.0
