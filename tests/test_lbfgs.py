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


def test_line_search_survives_a_flat_line():
    """A constant function along the search direction: the line search must end
    (no step through a zero-width bracket) and L-BFGS reports it."""
    def flat(x):
        return 1.0, np.full_like(x, 1e-3)
    r = vqe.lbfgs(flat, np.zeros(3), maxiter=5)
    assert r.reason in ("linesearch", "ftol", "maxiter")


def test_scan_comparison_counts_points_after_the_shared_ones():
    """pes_scan.compare: E_ref is the lower converged energy per point, an arm's
    cost is its first iteration within 1e-6 Ha of it, only points after the
    min_train shared ones are totalled, and the network's training is added in
    seconds_with_fit by the caller."""
    from paper_2606_28952_gb300 import pes_scan

    def pr(R, E_hist, t_hist, fev_hist, start="previous", fit=0.0):
        r = vqe.PointResult(R, start, E_hist[-1], len(E_hist) - 1, fev_hist[-1], t_hist[-1], list(E_hist),
                            list(t_hist), list(fev_hist), np.zeros(2), E_hist[0])
        r.fit_seconds = fit
        return r

    prev = [pr(0.5, [0.0, -1.0], [0.0, 1.0], [1, 3]),
            pr(0.6, [-0.9, -1.0000005, -1.0000009], [0.0, 0.5, 1.0], [1, 3, 5]),
            pr(0.7, [-0.8, -0.9], [0.0, 2.0], [1, 4])]
    warm = [prev[0],
            pr(0.6, [-1.0000008, -1.0000009], [0.0, 0.3], [3, 5], start="mlp", fit=0.1),
            pr(0.7, [-0.95, -1.2], [0.0, 1.5], [3, 8], start="mlp", fit=0.2)]
    rows, tot, reached = pes_scan.compare(prev, warm, min_train=1)
    assert rows[1]["E_ref"] == -1.0000009 and rows[2]["E_ref"] == -1.2
    # point 1: previous reaches -1.0000009 + 1e-6 at iteration 1 (0.5 s, 3 evaluations),
    # the network's start is already there (iteration 0)
    assert rows[1]["previous"]["to_target"] == {"iterations": 1, "evaluations": 3, "seconds": 0.5}
    assert rows[1]["mlp"]["to_target"] == {"iterations": 0, "evaluations": 3, "seconds": 0.0}
    # point 2: the previous arm never gets within 1e-6 of -1.2
    assert rows[2]["previous"]["to_target"] is None and reached["previous"] == 1 and reached["mlp"] == 2
    assert tot["previous"] == [1, 3, 0.5] and tot["mlp"] == [1, 11, 1.5]
