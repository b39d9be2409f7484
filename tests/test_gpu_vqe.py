"""GPU variational pieces vs the oracle: inner products, the fused adjoint
rotation, the product-ansatz energy and gradient, the BF16 tensor-core MLP
(forward, backward, Adam) and the gain of the learned warm start."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from oracle import vqe as ovqe
import workloads as w

pytestmark = pytest.mark.gpu

NORB = 4


@pytest.fixture(scope="module")
def ps():
    import torch
    import paper_2606_28952_gb300 as m
    assert torch.cuda.is_available()
    return m


def _tdt(name):
    import torch
    return torch.complex128 if name == "c128" else torch.complex64


def _dev(a, name):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", _tdt(name))


def _host(t):
    return t.cpu().numpy().astype(np.complex128)


# ----------------------------------------------------------------------------
# vdot
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("n", [0, 1, 255, 1000, (1 << 20) + 37])
def test_vdot(ps, dt, n):
    a = w.random_state(max(n, 1), 11)[:n]
    b = w.random_state(max(n, 1), 12)[:n]
    x, y = _dev(a, dt), _dev(b, dt)
    got = ps.vdot(x, y)
    ref = np.vdot(_host(x), _host(y))  # FP64 sum of the stored (possibly FP32) values
    assert abs(got - ref) <= 1e-13 * max(1.0, np.abs(_host(x)).sum() * 1.0)
    assert ps.vdot(x, y) == got  # fixed reduction order: same bits


# ----------------------------------------------------------------------------
# fused adjoint rotation
# ----------------------------------------------------------------------------
def _gens(norb, count):
    return [oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, p, q))
            for p, q in w.pair_double_ansatz(norb, count)]


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("norb", [4, 6])
def test_rotate_adjoint_matches_oracle(ps, dt, norb):
    import torch
    So = oracle.Sector.molecular(norb, norb // 2, norb // 2)
    S = ps.Sector.molecular(norb, norb // 2, norb // 2)
    tol = 1e-12 if dt == "c128" else 2e-6
    for k, (p, q) in enumerate(w.pair_double_ansatz(norb, 5)):
        Go = oracle.fermion_sum(2 * norb, w.pair_double_generator(norb, p, q))
        G = ps.PauliSum.jw_fermion(2 * norb, w.pair_double_generator(norb, p, q))
        phi, lam = _dev(w.random_state(S.dim, 30 + k), dt), _dev(w.random_state(S.dim, 60 + k), dt)
        phi0, lam0 = _host(phi), _host(lam)
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        theta = 0.37 * (k + 1)
        ps.rotate_adjoint(G, S, theta, phi, lam, out)
        mat = np.vdot(lam0, oracle.apply(So, Go, phi0))
        got = complex(out[0].item(), out[1].item())
        assert abs(got - mat) <= tol * max(1.0, abs(mat)), (p, q)
        assert np.linalg.norm(_host(phi) - oracle.rotate(So, Go, theta, phi0)) <= tol
        assert np.linalg.norm(_host(lam) - oracle.rotate(So, Go, theta, lam0)) <= tol


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_pair_listed_rotation_single_excitations(ps, dt):
    """Rotations whose X mask lies in the low half only (alpha excitations), the
    high half only (beta) or both (pair doubles), on an open-shell single-block
    sector: the pair-listed kernel against the oracle, forward and adjoint."""
    import torch
    norb, na, nb = 6, 3, 2
    So = oracle.Sector.molecular(norb, na, nb)
    S = ps.Sector.molecular(norb, na, nb)
    tol = 1e-12 if dt == "c128" else 2e-6
    gens = [w.single_generator(norb, p, q, spin) for (p, q, spin) in [(0, 4, 0), (1, 5, 1), (2, 3, 0), (0, 5, 1)]]
    gens += [w.pair_double_generator(norb, 1, 4)]
    for k, terms in enumerate(gens):
        Go = oracle.fermion_sum(2 * norb, terms)
        G = ps.PauliSum.jw_fermion(2 * norb, terms)
        phi0 = w.random_state(S.dim, 70 + k)
        lam0 = w.random_state(S.dim, 90 + k)
        phi, lam = _dev(phi0, dt), _dev(lam0, dt)
        ph_in, la_in = _host(phi), _host(lam)
        th = 0.3 + 0.2 * k
        ps.rotate(G, S, th, phi)
        assert np.linalg.norm(_host(phi) - oracle.rotate(So, Go, th, ph_in)) <= tol, k
        assert G.status() == 0
        phi = _dev(phi0, dt)
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        ps.rotate_adjoint(G, S, -th, phi, lam, out)
        mat = np.vdot(la_in, oracle.apply(So, Go, ph_in))
        assert abs(complex(out[0].item(), out[1].item()) - mat) <= tol * max(1.0, abs(mat)), k
        assert np.linalg.norm(_host(lam) - oracle.rotate(So, Go, -th, la_in)) <= tol, k


def test_rotate_seq_is_the_sequence_of_rotations(ps):
    norb = 6
    S = ps.Sector.molecular(norb, 3, 3)
    pairs = w.pair_double_ansatz(norb, 7)
    Gs = [ps.PauliSum.jw_fermion(2 * norb, w.pair_double_generator(norb, p, q)) for p, q in pairs]
    th = np.linspace(-0.5, 0.9, len(Gs))
    a = _dev(w.random_state(S.dim, 4), "c128")
    b = a.clone()
    ps.rotate_seq(Gs, S, th, a)
    for G, t in zip(Gs, th):
        ps.rotate(G, S, t, b)
    assert bool((a == b).all())


# ----------------------------------------------------------------------------
# energy and gradient of the product ansatz
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_energy_gradient_matches_oracle(ps, dt):
    from paper_2606_28952_gb300.vqe import EnergyGradient, ProductAnsatz
    h0, h1, g0 = w.pes_integrals(NORB, w.PES_SEED)
    h, g = w.pes_point(h0, h1, g0, 1.3)
    Ho = oracle.jw_hamiltonian(NORB, h, g, eps_drop=1e-12)
    So = oracle.Sector.molecular(NORB, 2, 2)
    count = 9
    gens_o = _gens(NORB, count)
    ref = int(So.index(oracle.hf_config(NORB, 2, 2))[0])
    S = ps.Sector.molecular(NORB, 2, 2)
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    ans = ps.vqe.ProductAnsatz.pair_doubles(NORB, w.pair_double_ansatz(NORB, count), S, oracle.hf_config(NORB, 2, 2))
    assert ans.ref_index == ref
    eg = EnergyGradient(H, S, ans, dtype=_tdt(dt))
    for seed in range(3):
        theta = np.random.default_rng(seed).uniform(-0.8, 0.8, count)
        E, grad = eg(theta)
        Eo = ovqe.energy(So, Ho, gens_o, theta, ref)
        go = ovqe.gradient(So, Ho, gens_o, theta, ref)
        etol, gtol = (1e-12, 1e-11) if dt == "c128" else (1e-6, 2e-5)
        assert abs(E - Eo) <= etol * max(1.0, abs(Eo))
        assert np.abs(grad - go).max() <= gtol * max(1.0, np.abs(go).max())
        assert abs(eg.energy(theta) - E) <= etol


def test_energy_gradient_on_the_12_orbital_sector(ps):
    """Full-size sector (853,776 amplitudes): gradient vs central differences of
    the GPU's own FP64 energy, a property that holds at any size."""
    from paper_2606_28952_gb300.vqe import EnergyGradient, ProductAnsatz
    import torch
    norb = 12
    h, g = w.MOL24.integrals()
    H = ps.PauliSum.jw_molecular(h, g, eps_drop=1e-12)
    S = ps.Sector.molecular(norb, 6, 6)
    ans = ProductAnsatz.pair_doubles(norb, w.pair_double_ansatz(norb, 12), S, oracle.hf_config(norb, 6, 6))
    eg = EnergyGradient(H, S, ans, dtype=torch.complex128)
    theta = np.random.default_rng(3).uniform(-0.3, 0.3, ans.size)
    E, grad = eg(theta)
    step = 1e-5
    for k in (0, 5, 11):
        e = np.zeros_like(theta)
        e[k] = step
        fd = (eg.energy(theta + e) - eg.energy(theta - e)) / (2 * step)
        assert abs(fd - grad[k]) < 1e-7 * max(1.0, abs(grad[k]))


# ----------------------------------------------------------------------------
# BF16 tensor-core MLP
# ----------------------------------------------------------------------------
def _mlp_case(ps, in_dim, hid, out_dim, B, seed):
    import torch
    from paper_2606_28952_gb300.vqe import glorot_params
    net = ps.MLP(in_dim, hid, out_dim, max(B, 8))
    p = glorot_params(net.shapes(), seed)
    p[in_dim * hid:in_dim * hid + hid] = np.random.default_rng(seed + 1).normal(0, 0.1, hid)  # non-zero b1
    net.set_params(p)
    rng = np.random.default_rng(seed + 2)
    x = rng.uniform(-1, 1, (B, in_dim)).astype(np.float32)
    T = rng.normal(0, 1, (B, out_dim)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    Td = torch.from_numpy(T).cuda()
    return net, p, x, T, xd, Td


@pytest.mark.parametrize("shape", [(1, 256, 200, 40), (1, 256, 200, 1), (3, 64, 37, 19), (2, 24, 5, 17)])
def test_mlp_forward_backward_match_oracle(ps, shape):
    in_dim, hid, out_dim, B = shape
    net, p, x, T, xd, Td = _mlp_case(ps, in_dim, hid, out_dim, B, 7)
    y = net.forward(xd).cpu().numpy()
    _, _, Yo = omlp.forward(p.astype(np.float64), x, in_dim, hid, out_dim, bf16=True)
    assert np.abs(y - Yo).max() <= 2e-3 * max(1.0, np.abs(Yo).max())
    loss, g = net.backward(xd, Td, want_grads=True)
    Lo, go = omlp.loss_and_grad(p.astype(np.float64), x, T, in_dim, hid, out_dim, bf16=True)
    assert abs(loss.item() - Lo) <= 2e-3 * max(1e-3, abs(Lo))
    g = g.cpu().numpy()
    # per block of the parameter vector, relative to that block's scale
    off = 0
    for name, shp in net.shapes():
        n = int(np.prod(shp))
        a, b = g[off:off + n], go[off:off + n]
        assert np.abs(a - b).max() <= 1e-2 * max(np.abs(b).max(), 1e-6), name
        off += n
    # and close to the exact FP64 gradient at BF16 accuracy
    _, gx = omlp.loss_and_grad(p.astype(np.float64), x, T, in_dim, hid, out_dim)
    assert np.linalg.norm(g - gx) <= 3e-2 * np.linalg.norm(gx)


def test_mlp_adam_step_matches_oracle(ps):
    net, p, x, T, xd, Td = _mlp_case(ps, 1, 64, 20, 12, 3)
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    wts = p.astype(np.float64)
    for t in range(1, 4):
        _, g = net.backward(xd, Td, want_grads=True)
        g = g.cpu().numpy().astype(np.float64)
        net.adam_step(1e-2, t)
        wts, m, v = omlp.adam(wts, g, m, v, 1e-2, t)
        assert np.abs(net.get_params() - wts).max() <= 1e-5 * max(1.0, np.abs(wts).max())


def test_mlp_train_call_equals_single_steps(ps):
    """pauli_mlp_train(steps) runs exactly the kernels of steps x (backward + adam),
    its first steps - 1 steps from a replayed graph: bit for bit the single steps,
    also on a second call that outgrows the first call's table (graph captured
    again) and a third with another learning rate."""
    net_a, p, x, T, xd, Td = _mlp_case(ps, 1, 64, 20, 12, 5)
    net_b, *_ = _mlp_case(ps, 1, 64, 20, 12, 5)
    t = 0
    for steps, lr in ((7, 3e-3), (12, 3e-3), (5, 1e-3)):
        la = net_a.train(xd, Td, steps, lr, t)
        for _ in range(steps):
            t += 1
            lb = net_b.backward(xd, Td)
            net_b.adam_step(lr, t)
        assert np.array_equal(net_a.get_params(), net_b.get_params()), (steps, lr)
        assert la.item() == lb.item()


def test_mlp_training_fits_a_smooth_map(ps):
    """Adam on the GPU fits theta(R) = a sin(R) + b R over 20 points."""
    import torch
    from paper_2606_28952_gb300.vqe import WarmStart
    rng = np.random.default_rng(0)
    a, b = rng.normal(0, 0.3, 50), rng.normal(0, 0.1, 50)
    ws = WarmStart(50, (0.5, 3.0), hidden=256, max_points=32, seed=1, window=32)
    Rs = np.linspace(0.5, 3.0, 20)
    for R in Rs:
        ws.add(R, a * np.sin(R) + b * R)
    l0 = None
    net = ws.net
    loss = ws.fit(steps=1, lr=1e-3)
    l0 = loss
    loss = ws.fit(steps=1500, lr=1e-3)
    assert loss < 2e-3 * l0
    R = 1.37
    assert np.abs(ws.predict(R) - (a * np.sin(R) + b * R)).max() < 0.05 * np.abs(a).max()


def test_mlp_rejects_bad_arguments(ps):
    import torch
    with pytest.raises(ps.PauliError):
        ps.MLP(0, 256, 10, 4)
    net = ps.MLP(1, 16, 4, 4)
    with pytest.raises(ValueError):
        net.forward(torch.zeros(5, 1, device="cuda"))
    with pytest.raises(ps.PauliError):
        net.adam_step(1e-3, 0)


# ----------------------------------------------------------------------------
# what the learned warm start gains
# ----------------------------------------------------------------------------
def test_learned_warm_start_gains_over_previous_point(ps):
    """A 14-point scan of the 12-qubit analog (6 orbitals, (3a,3b), 200 pair
    doubles): after 3 training points the network's starting angles reach the
    converged energy to 1e-6 Ha in fewer L-BFGS iterations, in total over the
    remaining points, than the previous point's angles."""
    from paper_2606_28952_gb300 import pes_scan
    out = pes_scan.run(norb=6, npoints=14, count=200, dtype="c128", min_train=3, fit_steps=1500, maxiter=300)
    prev, mlp = out["previous_start"], out["mlp_start"]
    assert mlp["reached"] == out["points_compared"]
    assert mlp["mlp_starts"] >= out["points_compared"] // 2
    assert mlp["iterations"] < prev["iterations"]
    assert mlp["evaluations"] < prev["evaluations"]
