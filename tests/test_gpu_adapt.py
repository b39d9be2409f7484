"""Operator-pool gradients (pauli_pool_gradients) and the ADAPT-VQE driver
against the oracle's commutator expectations <psi|[H, A_k]|psi>.

Tolerance: each gradient is a sum of products bounded by 2 ||H psi|| ||G_k psi||
(Cauchy-Schwarz); the error bound is 1e-12 (complex128) and 1e-5 (complex64)
of that scale, with the oracle run on the dtype-rounded psi and H psi."""
import numpy as np
import pytest

import oracle
from oracle import dense, vqe as ovqe
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


def _check_pool(ps, S, So, R, gens_dev, gens_or, psi, dt):
    import torch
    xin = _rounded(psi, dt)
    hin = _rounded(oracle.apply(So, R, xin), dt)
    # the oracle's commutator form on the same (rounded) psi; the GPU gets the rounded H psi
    ref = ovqe.pool_gradients(So, R, gens_or, xin)
    hn = np.linalg.norm(hin)
    scale = np.array([2 * hn * np.linalg.norm(oracle.apply(So, G, xin)) for G in gens_or])
    pool = ps.Pool(gens_dev, S)
    x = torch.from_numpy(xin).to("cuda", _tdt(dt))
    hx = torch.from_numpy(hin).to("cuda", _tdt(dt))
    g1 = pool.gradients(x, hx).cpu().numpy()
    g2 = pool.gradients(x, hx).cpu().numpy()
    assert np.array_equal(g1, g2)  # fixed reduction order
    # complex64: the rounding of H psi itself moves the result by ~1e-7 of the scale
    tol = TOL[dt] * np.maximum(scale, 1e-30) + (1e-6 * scale if dt == "c64" else 0.0)
    bad = np.nonzero(np.abs(g1 - ref) > tol)[0]
    assert len(bad) == 0, (bad[:5], g1[bad[:5]], ref[bad[:5]])
    return g1, ref


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb,na,nb,generalized", [(6, 3, 3, False), (8, 4, 4, False), (5, 2, 3, True)])
def test_pool_gradients_molecular(ps, dt, norb, na, nb, generalized):
    """Single-block sectors: pair-listed generators in one launch, plus a
    diagonal (x = 0) generator that takes the per-target kernel."""
    h, g = w.molecular_integrals(norb, 3)
    R = oracle.jw_hamiltonian(norb, h, g, eps_drop=1e-12)
    So = oracle.Sector.molecular(norb, na, nb)
    S = ps.Sector.molecular(norb, na, nb)
    pool = w.uccsd_pool(norb, na, nb, generalized=generalized)
    rng = np.random.default_rng(norb)
    wts = rng.normal(size=2 * norb)
    diag = [(float(wts[p]), [(p, 1), (p, 0)]) for p in range(2 * norb)]
    terms = [t for _, t in pool] + [diag]
    gens_or = [oracle.fermion_sum(2 * norb, t) for t in terms]
    gens_dev = [ps.PauliSum.jw_fermion(2 * norb, t) for t in terms]
    psi = w.random_state(So.dim, 300 + norb)
    g1, ref = _check_pool(ps, S, So, R, gens_dev, gens_or, psi, dt)
    assert np.abs(ref).max() > 1e-2


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("kind", ["full", "sz0"])
def test_pool_gradients_lattice(ps, dt, kind):
    """Full space and several blocks (per-target kernel): bond X-groups, a single
    Pauli string and a diagonal generator of a 12-site chain."""
    n = 12
    x_, z_, cre, cim = w.xxz_terms(n, 1)
    H = oracle.build_sum(n, x_, z_, None, cre, cim)
    gens = []
    for i in (0, 4, 10):
        xm = (1 << i) | (1 << (i + 1))
        gens.append(([xm, xm], [0, xm], [0.7, -0.3]))           # a XX + b YY (letter form)
    gens.append(([0b101], [0b100], [0.5]))                        # X Z' X-type single string (Y on qubit 2)
    gens.append(([0, 0, 0], [1, 2, 6], [0.3, -0.8, 0.25]))       # diagonal
    if kind == "full":
        So, S = oracle.Sector.full(n), ps.Sector.full(n, 6)
    else:
        blocks = [(k, 6 - k) for k in range(7)]
        So, S = oracle.Sector(n, oracle.BLOCKS, 6, blocks), ps.Sector(n, ps.BLOCKS, 6, blocks)
        gens = gens[:3] + gens[4:]  # the single string changes Sz
    gens_or = [oracle.build_sum(n, np.array(a, np.uint64), np.array(b, np.uint64), None, np.array(c),
                                np.zeros(len(c))) for a, b, c in gens]
    gens_dev = [ps.PauliSum.from_terms(n, a, b, c) for a, b, c in gens]
    psi = w.random_state(So.dim, 55)
    _check_pool(ps, S, So, H, gens_dev, gens_or, psi, dt)


def test_pool_gradients_match_the_adjoint_step(ps):
    """The pool gradient of G at psi equals the last adjoint-sweep entry of the
    one-generator ansatz exp(-i 0 G) psi (2 Im <H psi|G psi>), on the 24-qubit
    molecule's pool (1,818 UCCSD generators, one launch)."""
    import torch
    h, g = w.MOL24.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(12, 6, 6)
    pool_terms = w.uccsd_pool(12, 6, 6)
    gens = [ps.PauliSum.jw_fermion(24, t) for _, t in pool_terms]
    P = ps.Pool(gens, S)
    psi = torch.from_numpy(w.random_state(S.dim, 12)).to("cuda")
    hpsi = torch.empty_like(psi)
    ps.expect(H, S, psi, hpsi_out=hpsi)
    grads = P.gradients(psi, hpsi).cpu().numpy()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for k in (0, 71, 72, 500, 1817):
        phi, lam = psi.clone(), hpsi.clone()
        ps.rotate_adjoint(gens[k], S, 0.0, phi, lam, out)
        assert abs(2 * out[1].item() - grads[k]) <= 1e-12 * max(1.0, abs(grads[k])) * 10, k


def test_adapt_vqe_12_qubits(ps):
    """ADAPT-VQE on the 12-qubit molecule with the UCCSD pool: the first
    selection is the oracle's largest |<HF|[H, A_k]|HF>|, energies fall
    monotonically from E_HF, and stay above the exact sector ground state."""
    from paper_2606_28952_gb300 import vqe
    h, g = w.MOL12.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(6, 3, 3)
    R = oracle.jw_hamiltonian(6, h, g, eps_drop=1e-12)
    So = oracle.Sector.molecular(6, 3, 3)
    pool_terms = w.uccsd_pool(6, 3, 3)
    gens = [ps.PauliSum.jw_fermion(12, t) for _, t in pool_terms]
    hf = oracle.hf_config(6, 3, 3)
    res = vqe.adapt_vqe(H, S, gens, hf, max_ops=8, grad_tol=1e-4)
    e_hf = oracle.hf_energy(6, h, g, 3, 3)
    assert abs(res.energies[0] - e_hf) < 1e-12
    assert all(b <= a + 1e-10 for a, b in zip(res.energies, res.energies[1:]))
    Hs = dense.sector_matrix(12, R.x, R.z, R.c, So.configs())
    e0 = np.linalg.eigvalsh(Hs)[0]
    assert res.energies[-1] >= e0 - 1e-9 and res.energies[-1] < e_hf - 1e-3
    # the first choice agrees with the oracle at the HF state
    psi_hf = np.zeros(So.dim, np.complex128)
    psi_hf[int(So.index(hf)[0])] = 1.0
    gens_or = [oracle.fermion_sum(12, t) for _, t in pool_terms]
    g_or = ovqe.pool_gradients(So, R, gens_or, psi_hf)
    assert abs(abs(g_or).max() - res.grad_norms[0]) < 1e-10
    assert abs(g_or[res.selected[0]]) >= abs(g_or).max() - 1e-10
