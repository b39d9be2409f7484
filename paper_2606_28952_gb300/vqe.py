"""Variational driver over the operator engine: a product ansatz of
single-group Pauli rotations (pair doubles, Sec. 3.2), its energy from
pauli_expect and its exact gradient from one adjoint sweep of fused
rotate-and-contract launches, an L-BFGS optimiser, and the learned warm start
(an MLP trained on the converged angles of earlier geometries, Sec. 4) for a
scan over a bond coordinate.

Everything that touches a state vector runs in the library's kernels; the
optimiser works on the K angles on the host (K = 200 numbers per step).
"""
from __future__ import annotations

import copy
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import MLP, PauliSum, Pool, Sector, expect, expect_rows, rotate_adjoint, rotate_seq


# ---------------------------------------------------------------------------
# ansatz and energy / gradient
# ---------------------------------------------------------------------------
class ProductAnsatz:
    """psi(theta) = U_{K-1} ... U_0 |ref>, U_k = exp(-i theta_k G_k).

    ``generators`` is a list of K single-X-group Hermitian Pauli sums (repeats
    share one handle); ``ref_index`` the sector index of the reference
    configuration."""

    def __init__(self, generators, ref_index: int):
        self.generators = list(generators)
        self.ref_index = int(ref_index)

    @property
    def size(self) -> int:
        return len(self.generators)

    @classmethod
    def pair_doubles(cls, norb: int, pairs, sector: Sector, ref_config: int):
        from workloads import pair_double_generator  # generator recipe (fermionic monomials)
        cache = {}
        gens = []
        for p, q in pairs:
            if (p, q) not in cache:
                cache[(p, q)] = PauliSum.jw_fermion(2 * norb, pair_double_generator(norb, p, q), eps_drop=1e-14)
            gens.append(cache[(p, q)])
        import torch
        ref = int(sector.rank(torch.tensor([ref_config], dtype=torch.int64, device="cuda"))[0].item())
        if ref < 0:
            raise ValueError("the reference configuration is not in the sector")
        return cls(gens, ref)


class EnergyGradient:
    """E(theta) = <psi(theta)|H|psi(theta)> and dE/dtheta on one GPU.

    One evaluation: copy |ref>, K rotations, one pauli_expect that also keeps
    lam = H psi, then K fused adjoint launches (k = K-1 .. 0) that each add
    <lam|G_k|phi> to a device array and undo U_k on phi and lam; a single
    device-to-host copy brings E and the K gradient entries back.

    ``rows`` (sector indices, device int64): a set of configurations that every
    generator maps onto itself and that holds the reference, so psi(theta)
    vanishes off it.  Then pauli_expect_rows gives E and lam = P H psi (P the
    projector on the rows) from those rows alone; the rotations keep P lam and
    (1 - P) lam apart, and <lam|G_k|phi> only sees P lam, so the gradient is
    the same as with the full H psi."""

    def __init__(self, H: PauliSum, sector: Sector, ansatz: ProductAnsatz, dtype=None, device="cuda", rows=None):
        import torch
        self.torch = torch
        self.H, self.s, self.ansatz = H, sector, ansatz
        self.dtype = dtype or torch.complex128
        K = ansatz.size
        self.ref = torch.zeros(sector.dim, dtype=self.dtype, device=device)
        self.ref[ansatz.ref_index] = 1.0
        self.psi = torch.empty_like(self.ref)
        self.lam = torch.zeros_like(self.ref) if rows is not None else torch.empty_like(self.ref)
        self.rows = rows
        self.res = torch.zeros(4 + 2 * K, dtype=torch.float64, device=device)
        self.evals = 0

    def _expect(self, hpsi_out=None):
        if self.rows is None:
            expect(self.H, self.s, self.psi, hpsi_out=hpsi_out, result=self.res[:4])
        else:
            if hpsi_out is not None:
                # entries off the rows stay zero: the adjoint sweep rotates zeros into zeros
                hpsi_out.zero_()
            expect_rows(self.H, self.s, self.psi, self.rows, hpsi_out=hpsi_out, result=self.res[:4])

    def state(self, theta):
        self.psi.copy_(self.ref)
        rotate_seq(self.ansatz.generators, self.s, np.asarray(theta, dtype=np.float64), self.psi)
        return self.psi

    def energy(self, theta) -> float:
        self.state(theta)
        self._expect()
        self.evals += 1
        return float(self.res[0].item())

    def __call__(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        self.state(theta)
        self._expect(hpsi_out=self.lam)
        gens = self.ansatz.generators
        for k in range(len(gens) - 1, -1, -1):
            rotate_adjoint(gens[k], self.s, -float(theta[k]), self.psi, self.lam, self.res[4 + 2 * k:6 + 2 * k])
        host = self.res.cpu().numpy()
        self.evals += 1
        return float(host[0]), 2.0 * host[5::2].copy()


# ---------------------------------------------------------------------------
# L-BFGS with a strong-Wolfe line search
# ---------------------------------------------------------------------------
@dataclass
class LbfgsResult:
    x: np.ndarray
    f: float
    g: np.ndarray
    nit: int
    nfev: int
    reason: str
    f_hist: list = field(default_factory=list)    # f after each iteration (index 0: start)
    t_hist: list = field(default_factory=list)    # wall time (s) at each entry of f_hist
    fev_hist: list = field(default_factory=list)  # evaluations used at each entry of f_hist


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic through (a, fa, ga), (b, fb, gb), or None."""
    if a == b:
        return None
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - ga * gb
    if disc < 0:
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = gb - ga + 2.0 * d2
    if den == 0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def _armijo_fails(fa, f0, a, g0, c1):
    # sufficient decrease, with room for the rounding of f itself
    return fa > f0 + c1 * a * g0 + 4.0 * np.finfo(float).eps * abs(f0)


def _zoom(phi, lo, hi, f0, g0, c1, c2, maxit=30):
    """Bracket-shrinking stage of the strong-Wolfe search (lo, hi: (a, f, g, x-data))."""
    for _ in range(maxit):
        a_lo, f_lo, g_lo, _ = lo
        a_hi, f_hi, g_hi, _ = hi
        if abs(a_hi - a_lo) < 1e-14 * max(1.0, abs(a_lo)):
            break  # the bracket has collapsed
        a = _cubic_min(a_lo, f_lo, g_lo, a_hi, f_hi, g_hi)
        left, right = min(a_lo, a_hi), max(a_lo, a_hi)
        w = right - left
        if a is None or not (left + 0.1 * w <= a <= right - 0.1 * w):
            a = 0.5 * (a_lo + a_hi)
        fa, ga, data = phi(a)
        if _armijo_fails(fa, f0, a, g0, c1) or fa >= f_lo:
            hi = (a, fa, ga, data)
        else:
            if abs(ga) <= -c2 * g0:
                return a, fa, ga, data
            if ga * (a_hi - a_lo) >= 0:
                hi = lo
            lo = (a, fa, ga, data)
        if abs(hi[0] - lo[0]) < 1e-14 * max(1.0, abs(lo[0])):
            break
    return lo


def line_search_wolfe(phi, f0, g0, a1=1.0, c1=1e-4, c2=0.9, amax=50.0, maxit=20):
    """Step a with f(a) <= f0 + c1 a g0 and |f'(a)| <= c2 |g0| (strong Wolfe);
    phi(a) -> (f, f', data).  Returns (a, f, f', data) or None."""
    prev = (0.0, f0, g0, None)
    a = a1
    for i in range(maxit):
        fa, ga, data = phi(a)
        if _armijo_fails(fa, f0, a, g0, c1) or (i > 0 and fa >= prev[1]):
            return _zoom(phi, prev, (a, fa, ga, data), f0, g0, c1, c2)
        if abs(ga) <= -c2 * g0:
            return a, fa, ga, data
        if ga >= 0:
            return _zoom(phi, (a, fa, ga, data), prev, f0, g0, c1, c2)
        prev = (a, fa, ga, data)
        if a >= amax:
            break  # the step cap is reached: take the last step
        a = min(2.0 * a, amax)
    return prev if prev[3] is not None else None


def lbfgs(fg, x0, m: int = 20, gtol: float = 1e-6, ftol: float = 1e-12, patience: int = 5, maxiter: int = 500,
          max_step: float = 0.5, stop=None) -> LbfgsResult:
    """Minimise f with gradient fg(x) -> (f, g).

    Two-loop recursion over the last m pairs, initial scaling s'y / y'y,
    strong-Wolfe steps.  Stops at max|g| <= gtol, at `patience` consecutive
    iterations with f decreasing by <= ftol max(1, |f|), at maxiter, or when
    stop(f, nit) returns True.  The first trial step is capped at max_step in
    the infinity norm."""
    t0 = time.perf_counter()
    x = np.array(x0, dtype=np.float64)
    f, g = fg(x)
    nfev = 1
    S, Y, RHO = [], [], []
    res = LbfgsResult(x, f, g, 0, nfev, "maxiter", [f], [time.perf_counter() - t0], [1])
    small = 0
    for it in range(1, maxiter + 1):
        if np.max(np.abs(g)) <= gtol:
            res.reason = "gtol"
            break
        q = g.copy()
        alphas = []
        for s, y, rho in zip(reversed(S), reversed(Y), reversed(RHO)):
            a = rho * np.dot(s, q)
            alphas.append(a)
            q -= a * y
        gamma = np.dot(S[-1], Y[-1]) / np.dot(Y[-1], Y[-1]) if S else 1.0
        r = gamma * q
        for (s, y, rho), a in zip(zip(S, Y, RHO), reversed(alphas)):
            b = rho * np.dot(y, r)
            r += s * (a - b)
        d = -r
        gd = float(np.dot(g, d))
        if gd >= 0:  # not a descent direction: restart from steepest descent
            S, Y, RHO = [], [], []
            d = -g
            gd = float(np.dot(g, d))
        dmax = float(np.max(np.abs(d)))
        a1 = min(1.0, max_step / dmax) if dmax > 0 else 1.0
        n0 = nfev

        def phi(a):
            nonlocal nfev
            xa = x + a * d
            fa, ga = fg(xa)
            nfev += 1
            return fa, float(np.dot(ga, d)), (xa, ga)

        ls = line_search_wolfe(phi, f, gd, a1=a1)
        if ls is None or ls[3] is None:
            res.reason = "linesearch"
            break
        a, fa, _, (xa, ga) = ls
        s_vec, y_vec = xa - x, ga - g
        sy = float(np.dot(s_vec, y_vec))
        if sy > 1e-16 * float(np.dot(y_vec, y_vec)):
            S.append(s_vec)
            Y.append(y_vec)
            RHO.append(1.0 / sy)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
                RHO.pop(0)
        df = f - fa
        x, f, g = xa, fa, ga
        res.nit = it
        res.f_hist.append(f)
        res.t_hist.append(time.perf_counter() - t0)
        res.fev_hist.append(nfev)
        small = small + 1 if df <= ftol * max(1.0, abs(f)) else 0
        if small >= patience:
            res.reason = "ftol"
            break
        if stop is not None and stop(f, it):
            res.reason = "stop"
            break
        if nfev - n0 == 0:
            break
    res.x, res.f, res.g, res.nfev = x, f, g, nfev
    return res


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# ADAPT-VQE: operator selection by pool gradients (Sec. 3.3)
# ---------------------------------------------------------------------------
@dataclass
class AdaptResult:
    energies: list          # E after each re-optimisation (index 0: the reference)
    selected: list          # pool indices in the order they were appended
    grad_norms: list        # max |g_k| over the pool before each selection
    theta: np.ndarray
    reason: str


def adapt_vqe(H: PauliSum, sector: Sector, pool_gens, ref_config: int, max_ops: int = 20, grad_tol: float = 1e-3,
              dtype=None, gtol: float = 1e-7, maxiter: int = 200) -> AdaptResult:
    """ADAPT-VQE over a pool of single-group generators: from the reference
    configuration, repeatedly compute every pool gradient g_k = <psi|[H, A_k]|psi>
    in one pauli_pool_gradients pass (H psi from pauli_expect), append the
    generator with the largest |g_k| to the product ansatz (angle 0) and
    re-optimise all angles with L-BFGS (adjoint gradients); stop when
    max |g_k| < grad_tol or after max_ops generators."""
    import torch
    dtype = dtype or torch.complex128
    ref = int(sector.rank(torch.tensor([ref_config], dtype=torch.int64, device="cuda"))[0].item())
    if ref < 0:
        raise ValueError("the reference configuration is not in the sector")
    pool = Pool(pool_gens, sector)
    psi = torch.zeros(sector.dim, dtype=dtype, device="cuda")
    hpsi = torch.empty_like(psi)
    res = torch.empty(4, dtype=torch.float64, device="cuda")
    chosen, theta = [], np.zeros(0)
    out = AdaptResult([], [], [], theta, "max_ops")
    for it in range(max_ops + 1):
        psi.zero_()
        psi[ref] = 1.0
        if chosen:
            rotate_seq([pool_gens[k] for k in chosen], sector, theta, psi)
        expect(H, sector, psi, hpsi_out=hpsi, result=res)
        if it == 0:
            out.energies.append(float(res[0].item()))
        g = pool.gradients(psi, hpsi).cpu().numpy()
        k = int(np.argmax(np.abs(g)))
        out.grad_norms.append(float(abs(g[k])))
        if abs(g[k]) < grad_tol:
            out.reason = "grad_tol"
            break
        if it == max_ops:
            break
        chosen.append(k)
        theta = np.concatenate([theta, [0.0]])
        eg = EnergyGradient(H, sector, ProductAnsatz([pool_gens[j] for j in chosen], ref), dtype=dtype)
        r = lbfgs(eg, theta, gtol=gtol, maxiter=maxiter)
        theta = r.x
        out.energies.append(float(r.f))
    out.selected = chosen
    out.theta = theta
    pool.close()
    return out


def glorot_params(shapes, seed: int) -> np.ndarray:
    """Seeded initial parameter vector: uniform Glorot weights, zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shp in shapes:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / (shp[0] + shp[1]))
            out.append(rng.uniform(-lim, lim, size=shp).reshape(-1))
        else:
            out.append(np.zeros(shp).reshape(-1))
    return np.concatenate(out).astype(np.float32)


class WarmStart:
    """R -> theta regression on the converged angles of earlier points.

    Inputs are the bond coordinate mapped to [-1, 1] over the scan range;
    targets are the angles standardised per component over the training set,
    (theta_j - mean_j) / std_j, so the network's BF16 resolution applies to
    how the angles vary along the scan rather than to their size.  The network
    is trained on the GPU (pauli_mlp_* kernels, full batch over the most
    recent `window` points, Adam) and keeps its weights from one point to the
    next.  ``step`` gives the start used by the
    scan: the previous converged angles moved by the change the network
    predicts between the two geometries, theta_prev + f(R) - f(R_prev), which
    cancels the network's own offset at R_prev."""

    def __init__(self, n_theta: int, r_range, hidden: int = 256, max_points: int = 64, seed: int = 0,
                 window: int = 10):
        import torch
        self.torch = torch
        self.window = int(window)
        self.net = MLP(1, hidden, n_theta, max(2, min(max_points, self.window)))
        self.net.set_params(glorot_params(self.net.shapes(), seed))
        self.r0, self.r1 = float(r_range[0]), float(r_range[1])
        self.R, self.T = [], []
        self.mu = np.zeros(n_theta)
        self.sd = np.ones(n_theta)
        self.t = 0
        self.loss = float("nan")

    def _x(self, R):
        return 2.0 * (np.asarray(R, dtype=np.float64) - self.r0) / (self.r1 - self.r0) - 1.0

    def add(self, R: float, theta):
        self.R.append(float(R))
        self.T.append(np.asarray(theta, dtype=np.float64))

    def fit(self, steps: int = 1500, lr: float = 1e-3) -> float:
        """Adam on the most recent `window` points (a kink of the angle curve
        leaves the training set after `window` further points)."""
        torch = self.torch
        T = np.stack(self.T[-self.window:])
        Rs = self.R[-self.window:]
        self.mu = T.mean(axis=0)
        self.sd = np.maximum(T.std(axis=0), 1e-9)
        x = torch.tensor(self._x(Rs), dtype=torch.float32, device="cuda").reshape(-1, 1).contiguous()
        y = torch.tensor((T - self.mu) / self.sd, dtype=torch.float32, device="cuda").contiguous()
        loss = self.net.train(x, y, steps, lr, self.t)
        self.t += steps
        self.loss = float(loss.item())
        return self.loss

    def _f(self, Rs):
        torch = self.torch
        x = torch.tensor(self._x(Rs), dtype=torch.float32, device="cuda").reshape(-1, 1).contiguous()
        return self.net.forward(x).cpu().numpy().astype(np.float64)

    def predict(self, R: float) -> np.ndarray:
        """The network's angles at R."""
        return self.mu + self.sd * self._f([R])[0]

    def step(self, R: float, R_prev: float, theta_prev) -> np.ndarray:
        """theta_prev + f(R) - f(R_prev)."""
        f = self._f([R, R_prev])
        return np.asarray(theta_prev, dtype=np.float64) + self.sd * (f[0] - f[1])


# ---------------------------------------------------------------------------
# scan over the bond coordinate
# ---------------------------------------------------------------------------
@dataclass
class PointResult:
    R: float
    start: str            # "previous", "mlp" or "reference"
    E: float
    nit: int
    nfev: int
    seconds: float
    f_hist: list
    t_hist: list
    fev_hist: list
    theta: np.ndarray
    E_start: float
    fit_seconds: float = 0.0
    fit_loss: float = float("nan")
    E_guess: float = float("nan")     # energy at the network's start
    E_previous: float = float("nan")  # energy at the previous point's angles
    reason: str = ""


def iterations_to(res: PointResult, E_target: float):
    """First (iteration, evaluations, seconds) with E <= E_target, else None."""
    for i, (f, t, n) in enumerate(zip(res.f_hist, res.t_hist, res.fev_hist)):
        if f <= E_target:
            return i, n, t
    return None


def scan(make_problem, points, n_theta: int, warm: WarmStart | None = None, min_train: int = 3,
         fit_steps: int = 150, lr: float = 1e-3, opt=None, log=None, reuse=()):
    """Optimise the ansatz at each point in order.  Without ``warm`` every point
    starts from the previous point's converged angles.  With it, once
    min_train points are known, the energies of the network's start
    warm.step(R, R_prev, theta_prev) and of the previous angles are computed
    (two energy-only evaluations, counted in nfev and the time) and L-BFGS
    starts from the lower one, so the previous angles are the fallback.
    ``reuse``: results of the first points taken as they are (a shared
    prefix that both kinds of start would compute identically).
    make_problem(R) -> EnergyGradient."""
    opt = dict(opt or {})
    out = []
    theta_prev = np.zeros(n_theta)
    R_prev = None
    for i, R in enumerate(points):
        if i < len(reuse):
            res = copy.copy(reuse[i])
        else:
            eg = make_problem(R)
            t0 = time.perf_counter()
            start, x0 = ("reference" if i == 0 else "previous"), theta_prev
            extra = 0
            e_guess = e_prev = float("nan")
            if warm is not None and len(warm.R) >= min_train:
                guess = warm.step(R, R_prev, theta_prev)
                e_guess, e_prev = eg.energy(guess), eg.energy(theta_prev)
                extra = 2
                if e_guess < e_prev:
                    start, x0 = "mlp", guess
            t_pre = time.perf_counter() - t0
            r = lbfgs(eg, x0, **opt)
            secs = time.perf_counter() - t0
            res = PointResult(R, start, r.f, r.nit, r.nfev + extra, secs, r.f_hist, [t + t_pre for t in r.t_hist],
                              [n + extra for n in r.fev_hist], r.x, r.f_hist[0])
            res.E_guess, res.E_previous = e_guess, e_prev
            res.reason = r.reason
        theta_prev, R_prev = res.theta, R
        if warm is not None:
            t1 = time.perf_counter()
            warm.add(R, res.theta)
            if len(warm.R) >= min_train:
                res.fit_loss = warm.fit(fit_steps, lr)
            res.fit_seconds = time.perf_counter() - t1
        out.append(res)
        if log:
            log(f"R={R:.4f} start={res.start:9s} E0={res.E_start:.8f} E={res.E:.10f} nit={res.nit} nfev={res.nfev} "
                f"{res.seconds:.2f}s ({res.reason}) fit={res.fit_loss:.2e} E(guess)-E={res.E_guess - res.E:.2e} "
                f"E(prev)-E={res.E_previous - res.E:.2e}")
    return out
