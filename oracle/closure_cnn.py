"""Periodic 3x3 convolution network, forward and backward in FP64 (oracle).

The learned closure has no counterpart in the paper; this is the plain
definition the GPU kernels are checked against.  One layer is the circular
cross-correlation
    y[o, i, j] = bias[o] + sum_{c, p, q} W[o, c, p, q] x[c, (i + p - 1) mod H, (j + q - 1) mod W]
with p, q in {0, 1, 2}; layers are separated by ReLU.  Input channels are
(Re u, Im u) on the coarse grid, output channels the correction to add.
Parity is pinned by finite differences; trained weights are parity unpinned.
"""
import numpy as np


def conv_forward(x, W, bias):
    """x (C, H, Wd), W (O, C, 3, 3), bias (O,) -> (O, H, Wd)."""
    O = W.shape[0]
    y = np.zeros((O,) + x.shape[1:]) + bias[:, None, None]
    for p in range(3):
        for q in range(3):
            xs = np.roll(x, shift=(1 - p, 1 - q), axis=(1, 2))    # xs[c,i,j] = x[c,i+p-1,j+q-1]
            y += np.tensordot(W[:, :, p, q], xs, axes=([1], [0]))
    return y


def conv_backward(x, W, gy):
    """Gradients (gx, gW, gbias) of sum(gy * conv_forward(x, W, b))."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for p in range(3):
        for q in range(3):
            xs = np.roll(x, shift=(1 - p, 1 - q), axis=(1, 2))
            gW[:, :, p, q] = np.tensordot(gy, xs, axes=([1, 2], [1, 2]))
            g = np.tensordot(W[:, :, p, q], gy, axes=([0], [0]))  # (C, H, Wd) at shifted positions
            gx += np.roll(g, shift=(p - 1, q - 1), axis=(1, 2))
    return gx, gW, gy.sum(axis=(1, 2))


def network_forward(x, params):
    """params = [(W0, b0), (W1, b1), ...]; ReLU between layers.  Returns output and activations."""
    acts = [x]
    h = x
    for li, (W, b) in enumerate(params):
        z = conv_forward(h, W, b)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h, acts


def network_backward(params, acts, gout):
    """Gradients of sum(gout * output) w.r.t. every (W, b), given the forward activations."""
    grads = [None] * len(params)
    g = gout
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li < len(params) - 1:
            g = g * (acts[li + 1] > 0.0)
        gx, gW, gb = conv_backward(acts[li], W, g)
        grads[li] = (gW, gb)
        g = gx
    return grads, g


def adamw_step(w, g, m, v, step, lr, beta1, beta2, eps, weight_decay):
    """One AdamW update (Adam moments, bias correction, decoupled weight decay); returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    w = w - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * w)
    return w, m, v


def mse(out, target):
    """Mean squared error and its gradient with respect to ``out``."""
    d = out - target
    return np.mean(d * d), 2.0 * d / d.size
