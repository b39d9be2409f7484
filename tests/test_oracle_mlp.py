"""Pins of the warm-start network oracle (oracle/mlp.py)."""
import numpy as np

from oracle import mlp

IN, HID, OUT, B = 1, 8, 5, 4


def _params(seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    n = IN * HID + HID + HID * HID + HID + HID * OUT + OUT
    return rng.normal(0, scale, n)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _params()
    x = rng.uniform(-1, 1, (B, IN))
    T = rng.normal(0, 1, (B, OUT))
    L, g = mlp.loss_and_grad(p, x, T, IN, HID, OUT)
    fd = np.zeros_like(p)
    h = 1e-6
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss_and_grad(p + e, x, T, IN, HID, OUT)[0] - mlp.loss_and_grad(p - e, x, T, IN, HID, OUT)[0]) / (2 * h)
    assert np.abs(g - fd).max() < 1e-8 * max(1.0, np.abs(g).max())


def test_zero_hidden_weights_closed_form():
    """W2 = W3 = 0: Y = b3, dW3 = outer(tanh(b2), sum_b dY), dW1 = db1 = dW2 = 0."""
    rng = np.random.default_rng(2)
    W1 = rng.normal(size=(IN, HID))
    b1 = rng.normal(size=HID)
    b2 = rng.normal(size=HID)
    b3 = rng.normal(size=OUT)
    p = np.concatenate([W1.ravel(), b1, np.zeros(HID * HID), b2, np.zeros(HID * OUT), b3])
    x = rng.uniform(-1, 1, (B, IN))
    T = rng.normal(size=(B, OUT))
    _, _, Y = mlp.forward(p, x, IN, HID, OUT)
    assert np.allclose(Y, np.broadcast_to(b3, (B, OUT)))
    L, g = mlp.loss_and_grad(p, x, T, IN, HID, OUT)
    assert abs(L - 0.5 * np.sum((b3 - T) ** 2) / B) < 1e-14
    dW1, db1, dW2, db2, dW3, db3 = mlp.unpack(g, IN, HID, OUT)
    dY = (b3 - T) / B
    assert np.allclose(db3, dY.sum(0), atol=1e-15)
    assert np.allclose(dW3, np.outer(np.tanh(b2), dY.sum(0)), atol=1e-15)
    assert np.abs(dW1).max() == 0 and np.abs(db1).max() == 0 and np.abs(dW2).max() == 0 and np.abs(db2).max() == 0


def test_first_adam_step_is_a_signed_step():
    g = np.array([3.0, -1e-3, 0.25, 0.0])
    w0 = np.ones(4)
    w1, m, v = mlp.adam(w0, g, np.zeros(4), np.zeros(4), lr=0.01, t=1)
    assert np.allclose(w1, w0 - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)
    assert np.allclose(w1[:3], w0[:3] - 0.01 * np.sign(g[:3]), atol=1e-7)


def test_bf16_rounding_is_nearest_even():
    one = 1.0
    u = 2.0 ** -7  # bfloat16 spacing at 1
    cases = {
        one: one,
        one + u / 2: one,                     # tie, 1.0 is even
        one + 1.5 * u: one + 2 * u,           # tie, rounds to the even neighbour
        one + u / 2 + 2.0 ** -20: one + u,    # just above the tie
        -3.0: -3.0,
        1e-3: 131 / 128 * 2.0 ** -10,         # 1.024 x 2^-10, 1.024 x 128 = 131.07 -> 131
    }
    for a, b in cases.items():
        assert mlp.bf16_round(np.array([a]))[0] == b, a


def test_bf16_emulation_changes_results_only_at_bf16_scale():
    rng = np.random.default_rng(3)
    p = _params(4)
    x = rng.uniform(-1, 1, (B, IN))
    T = rng.normal(0, 1, (B, OUT))
    _, g = mlp.loss_and_grad(p, x, T, IN, HID, OUT)
    _, gq = mlp.loss_and_grad(p, x, T, IN, HID, OUT, bf16=True)
    d = np.abs(g - gq).max() / np.abs(g).max()
    assert 1e-5 < d < 3e-2


def test_adam_recurrence_over_many_steps():
    """Adam's moments carried across steps.  With a constant gradient g the
    moments are m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so every
    bias-corrected step is -lr g / (|g| + eps); with a gradient that flips sign
    every step, m_t = (1 - b1) g (-1)^(t-1) (1 - (-b1)^t) / (1 + b1)
    (a geometric series) while v_t keeps the constant-gradient value."""
    b1, b2, lr, eps = 0.9, 0.999, 0.01, 1e-8
    g = np.array([2.0, -0.5, 1e-3, 7.0])
    w, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    T = 25
    for t in range(1, T + 1):
        w, m, v = mlp.adam(w, g, m, v, lr=lr, t=t, b1=b1, b2=b2, eps=eps)
        assert np.allclose(m, (1 - b1 ** t) * g, rtol=1e-13, atol=0)
        assert np.allclose(v, (1 - b2 ** t) * g * g, rtol=1e-12, atol=0)
    assert np.allclose(w, -T * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
    m, v = np.zeros(4), np.zeros(4)
    w = np.zeros(4)
    for t in range(1, T + 1):
        gt = g * (-1) ** (t - 1)
        w, m, v = mlp.adam(w, gt, m, v, lr=lr, t=t, b1=b1, b2=b2, eps=eps)
        m_closed = (1 - b1) * g * (-1) ** (t - 1) * (1 - (-b1) ** t) / (1 + b1)
        assert np.allclose(m, m_closed, rtol=1e-12, atol=0)
        assert np.allclose(v, (1 - b2 ** t) * g * g, rtol=1e-12, atol=0)
