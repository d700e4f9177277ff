"""Pins for the oracle's periodic 3x3 convolution network (CPU only)."""
import numpy as np

from oracle import closure_cnn as cnn


def test_conv_forward_brute_force():
    g = np.random.default_rng(2)
    x = g.standard_normal((2, 5, 4))
    W = g.standard_normal((3, 2, 3, 3))
    b = g.standard_normal(3)
    y = cnn.conv_forward(x, W, b)
    C, H, Wd = x.shape
    for o in range(3):
        for i in range(H):
            for j in range(Wd):
                s = b[o]
                for c in range(C):
                    for p in range(3):
                        for q in range(3):
                            s += W[o, c, p, q] * x[c, (i + p - 1) % H, (j + q - 1) % Wd]
                assert abs(y[o, i, j] - s) < 1e-12


def test_network_gradients_finite_differences():
    g = np.random.default_rng(3)
    shapes = [(3, 2), (3, 3), (2, 3)]
    params = [(g.standard_normal((o, c, 3, 3)) * 0.5, g.standard_normal(o) * 0.1) for o, c in shapes]
    x = g.standard_normal((2, 5, 6))
    gout = g.standard_normal((2, 5, 6))
    out, acts = cnn.network_forward(x, params)
    grads, gx = cnn.network_backward(params, acts, gout)
    f = lambda ps, xx: np.sum(gout * cnn.network_forward(xx, ps)[0])
    h = 1e-6
    for li in range(len(params)):
        for which in (0, 1):
            arr = params[li][which]
            for idx in [tuple(g.integers(0, s) for s in arr.shape) for _ in range(4)]:
                old = arr[idx]
                arr[idx] = old + h
                fp = f(params, x)
                arr[idx] = old - h
                fm = f(params, x)
                arr[idx] = old
                assert abs((fp - fm) / (2 * h) - grads[li][which][idx]) < 1e-6
    for idx in [(0, 1, 2), (1, 4, 5), (0, 0, 0)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        assert abs((f(params, xp) - f(params, xm)) / (2 * h) - gx[idx]) < 1e-6


def test_adamw_first_step_is_a_signed_step():
    # with zero moments, the first step moves each weight by lr * (g/|g| approximately + wd w)
    g = np.array([3.0, -0.5, 1e-3])
    w = np.array([1.0, 2.0, -1.0])
    w1, m, v = cnn.adamw_step(w, g, np.zeros(3), np.zeros(3), 1, 0.1, 0.9, 0.999, 1e-12, 0.01)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    assert np.allclose(w1, w - 0.1 * (np.sign(g) + 0.01 * w), atol=1e-9)


def test_mse_gradient_finite_difference():
    g = np.random.default_rng(4)
    out, tgt = g.standard_normal(12), g.standard_normal(12)
    loss, grad = cnn.mse(out, tgt)
    assert abs(loss - np.mean((out - tgt) ** 2)) < 1e-15
    h = 1e-6
    for i in range(12):
        o = out.copy(); o[i] += h
        lp, _ = cnn.mse(o, tgt)
        o[i] -= 2 * h
        lm, _ = cnn.mse(o, tgt)
        assert abs((lp - lm) / (2 * h) - grad[i]) < 1e-8


def test_adamw_constant_gradient_closed_form_over_many_steps():
    # With a constant gradient g and zero initial moments, m_t = (1 - beta1^t) g and
    # v_t = (1 - beta2^t) g^2 exactly, so the bias-corrected ratio is g / |g| at every step t
    # and each update is lr * (sign(g) + wd * w) up to eps.  A bias correction that drops the
    # exponent (beta instead of beta^t) passes step 1 but fails from step 2 on.
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    w = np.array([1.0, 2.0, -1.0, 0.25])
    m, v = np.zeros(4), np.zeros(4)
    lr, b1, b2, wd = 0.05, 0.9, 0.999, 0.01
    expect = w.copy()
    for t in range(1, 8):
        w, m, v = cnn.adamw_step(w, g, m, v, t, lr, b1, b2, 1e-14, wd)
        expect = expect - lr * (np.sign(g) + wd * expect)
        assert np.allclose(m, (1 - b1 ** t) * g, rtol=1e-14, atol=0)
        assert np.allclose(v, (1 - b2 ** t) * g * g, rtol=1e-13, atol=0)
        assert np.allclose(w, expect, rtol=0, atol=1e-9), t
