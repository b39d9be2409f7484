"""Host-side optimiser of the variational driver: L-BFGS with strong-Wolfe steps."""
import numpy as np

from paper_2606_28952_gb300 import vqe


def _rosen(x):
    f = np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2)
    g = np.zeros_like(x)
    g[:-1] = -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2 * (1 - x[:-1])
    g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
    return f, g


def test_rosenbrock():
    for n in (2, 10):
        x0 = np.full(n, -1.2)
        x0[1::2] = 1.0
        r = vqe.lbfgs(_rosen, x0, gtol=1e-9, maxiter=2000, max_step=1e9)
        assert np.abs(r.x - 1).max() < 1e-6, (n, r.reason, r.x)
        assert r.nit < 400


def test_quadratic_reaches_the_exact_minimiser():
    rng = np.random.default_rng(0)
    n = 30
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(np.logspace(0, 2, n)) @ Q.T
    b = rng.normal(size=n)
    r = vqe.lbfgs(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.zeros(n), gtol=1e-7, maxiter=500,
                  max_step=1e9, ftol=0.0)
    # |x - x*| <= |g| / lambda_min = |g| for this spectrum
    assert np.abs(r.x - np.linalg.solve(A, b)).max() < 1e-6
    assert r.reason == "gtol"
    # histories are monotone and consistent
    assert all(a >= b for a, b in zip(r.f_hist, r.f_hist[1:]))
    assert len(r.f_hist) == r.nit + 1 == len(r.fev_hist)


def test_line_search_returns_a_strong_wolfe_step():
    f = lambda a: (np.cos(3 * a) + 0.1 * (a - 2) ** 2, -3 * np.sin(3 * a) + 0.2 * (a - 2))
    # search along +1 from a point where the slope is negative
    a0 = 0.3
    fa0, ga0 = f(a0)
    assert ga0 < 0
    a, fa, ga, _ = vqe.line_search_wolfe(lambda a: (f(a0 + a)[0], f(a0 + a)[1], a), fa0, ga0, a1=1.0)
    assert fa <= fa0 + 1e-4 * a * ga0
    assert abs(ga) <= 0.9 * abs(ga0)


def test_stop_callback_and_history_times():
    r = vqe.lbfgs(_rosen, np.array([-1.2, 1.0]), stop=lambda f, it: it >= 3)
    assert r.reason == "stop" and r.nit == 3
    assert all(t1 >= t0 for t0, t1 in zip(r.t_hist, r.t_hist[1:]))
