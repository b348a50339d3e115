"""Pins of the training oracle (oracle/mlp.py: train_loss_grads, adam_update)
to values fixed independently of it: central finite differences of the loss
of the plain FP64 network, a network whose loss and gradients are known in
closed form, the invariance of the device-arithmetic form on BF16-exact
values, and Adam's first step and constant-gradient steps in closed form."""
import numpy as np

from oracle import mlp

ROWS = (256, 256, 256, 32)


def _net(rng, scale=1.0):
    w = [rng.standard_normal((r, 256)) * np.sqrt(2.0 / 256) * scale for r in ROWS]
    w[3] *= 0.3
    b = [rng.standard_normal(r) * 0.1 for r in ROWS]
    return w, b


def test_gradients_match_central_differences():
    """The chain rule of the plain FP64 network against (L(p + h) - L(p - h)) / 2h
    on sampled weights and biases of every layer (a dropped term, a wrong
    sign, a transposed operand or an index slip each fails here)."""
    rng = np.random.default_rng(1)
    n_in, n_out, B = 23, 7, 9
    w, b = _net(rng)
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal((B, n_out))
    loss, gw, gb = mlp.train_loss_grads(w, b, x, t, rounding=False)
    h = 1e-6
    for layer in range(4):
        rows = n_out if layer == 3 else ROWS[layer]
        cols = n_in if layer == 0 else 256
        for _ in range(12):
            o, i = rng.integers(rows), rng.integers(cols)
            wp = [x_.copy() for x_ in w]
            wp[layer][o, i] += h
            lp = mlp.train_loss_grads(wp, b, x, t, rounding=False)[0]
            wp[layer][o, i] -= 2 * h
            lm = mlp.train_loss_grads(wp, b, x, t, rounding=False)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gw[layer][o, i]) <= 1e-6 * max(abs(fd), 1e-3), (layer, o, i)
        for _ in range(6):
            o = rng.integers(rows)
            bp = [x_.copy() for x_ in b]
            bp[layer][o] += h
            lp = mlp.train_loss_grads(w, bp, x, t, rounding=False)[0]
            bp[layer][o] -= 2 * h
            lm = mlp.train_loss_grads(w, bp, x, t, rounding=False)[0]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gb[layer][o]) <= 1e-6 * max(abs(fd), 1e-3), (layer, o)
    # unused inputs and outputs carry exactly zero gradient
    assert not np.any(gw[0][:, n_in:])
    assert not np.any(gw[3][n_out:]) and not np.any(gb[3][n_out:])
    assert loss > 0


def test_constant_network_closed_form():
    """Zero weights and hidden biases, output bias c: y = c for every row, so
    L = mean (c_o - t_ro)^2, dL/db3_o = 2 sum_r (c_o - t_ro) / (B n_out), and
    every other gradient is zero (the hidden activations are zero)."""
    rng = np.random.default_rng(2)
    n_in, n_out, B = 11, 5, 6
    w = [np.zeros((r, 256)) for r in ROWS]
    b = [np.zeros(r) for r in ROWS]
    c = np.zeros(32)
    c[:n_out] = [0.5, -1.25, 2.0, 0.0, 3.5]
    b[3] = c
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal((B, n_out))
    for rounding in (False, True):
        loss, gw, gb = mlp.train_loss_grads(w, b, x, t, rounding=rounding)
        assert np.isclose(loss, np.mean((c[:n_out] - t) ** 2), rtol=1e-14)
        want = np.zeros(32)
        want[:n_out] = 2.0 * (c[:n_out] - t).sum(axis=0) / (B * n_out)
        assert np.allclose(gb[3], want, rtol=1e-14, atol=0)
        for layer in range(4):
            assert not np.any(gw[layer])
        for layer in range(3):
            assert not np.any(gb[layer])


def test_device_form_equals_plain_form_on_bf16_exact_values():
    """Weights, inputs and every intermediate exactly representable in BF16
    (small dyadic values, one active path per unit): the rounded form
    reduces to the plain one."""
    n_in, n_out, B = 4, 2, 4            # B n_out a power of two: 2 d / (B n_out) stays exact
    w = [np.zeros((r, 256)) for r in ROWS]
    b = [np.zeros(r) for r in ROWS]
    for k in range(n_in):
        w[0][k, k] = 0.5
        w[1][k, k] = 2.0
        w[2][k, k] = 1.0
    w[3][0, :n_in] = [1.0, 0.5, 0.25, 0.0]
    w[3][1, :n_in] = [0.0, 1.0, -1.0, 2.0]
    x = np.array([[1.0, 2.0, -1.0, 0.5], [0.25, -2.0, 3.0, 1.0], [4.0, 0.5, 0.5, -0.5], [-1.0, 1.0, 2.0, 0.25]])
    t = np.array([[0.5, 1.0], [-1.0, 0.25], [2.0, 0.0], [0.75, -0.5]])
    a = mlp.train_loss_grads(w, b, x, t, rounding=False)
    r = mlp.train_loss_grads(w, b, x, t, rounding=True)
    assert a[0] == r[0]
    for layer in range(4):
        assert np.array_equal(a[1][layer], r[1][layer]) and np.array_equal(a[2][layer], r[2][layer])


def test_adam_first_and_constant_gradient_steps():
    """With m = v = 0, the bias-corrected moments of step 1 are g and g^2, so
    the step is -lr g / (|g| + eps); a gradient held constant keeps both
    corrected moments exactly g and g^2 at every later step."""
    g = np.array([1e-3, -2.0, 0.5, 0.0, -1e-9])
    p0 = np.array([0.1, -0.2, 0.3, 0.4, 0.5])
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 0.01
    step = -lr * g / (np.abs(g) + eps)
    p, m, v = p0.copy(), np.zeros(5), np.zeros(5)
    for t in range(1, 6):
        p_prev = p
        p, m, v = mlp.adam_update(p, g, m, v, t, lr, b1, b2, eps, wd)
        assert np.allclose(p, (p_prev + step) * (1.0 - lr * wd), rtol=1e-12, atol=1e-18), t
    q, _, _ = mlp.adam_update(p0, g, np.zeros(5), np.zeros(5), 1, lr, b1, b2, eps, wd, decay=False)
    assert np.allclose(q, p0 + step, rtol=1e-14, atol=0)
