"""Pins for the oracle's Ginzburg-Landau right-hand side and steppers (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import fourier
from oracle import ginzburg_landau as gl

L = 100.0


def _grid(M):
    X = -50.0 + L * np.arange(M) / M
    return X[:, None], X[None, :]


def _plane_wave(M, l0, l1, beta, gamma, t):
    k0, k1 = 2 * np.pi * l0 / L, 2 * np.pi * l1 / L
    k2 = k0 ** 2 + k1 ** 2
    A = np.sqrt(1 - k2)
    om = beta * k2 + gamma * (1 - k2)
    x, y = _grid(M)
    return A * np.exp(1j * (k0 * (x + 50) + k1 * (y + 50) - om * t))


@pytest.mark.parametrize("stepper", [gl.rk4_step, gl.if_rk4_step])
def test_plane_wave_fourth_order(stepper):
    # u = A exp(i(k.x - w t)), |A|^2 = 1 - |k|^2, w = beta|k|^2 + gamma(1 - |k|^2) is exact.
    M, beta, gamma, T = 12, 1.5, -0.5, 1.0
    u0 = fourier.c2c_forward(fourier.c2c_forward(_plane_wave(M, 2, 1, beta, gamma, 0.0), 0), 1)
    exact = fourier.c2c_forward(fourier.c2c_forward(_plane_wave(M, 2, 1, beta, gamma, T), 0), 1)
    errs = []
    for n in (10, 20):
        u = u0
        for _ in range(n):
            u = stepper(u, T / n, beta, gamma)
        errs.append(np.max(np.abs(u - exact)))
    assert errs[1] < 1e-5
    assert 12 < errs[0] / errs[1] < 20          # fourth order: ratio 2^4


def test_uniform_state_closed_form():
    # spatially uniform u: s = |u|^2 obeys s' = 2 s (1 - s); theta' = -gamma s.
    M, beta, gamma, T, n = 6, 1.5, 1.5, 0.5, 200
    s0, th0 = 0.09, 0.3
    uh = np.zeros((M, M), complex)
    uh[0, 0] = np.sqrt(s0) * np.exp(1j * th0)
    for _ in range(n):
        uh = gl.rk4_step(uh, T / n, beta, gamma)
    s = s0 * np.exp(2 * T) / (1 - s0 + s0 * np.exp(2 * T))
    th = th0 - 0.5 * gamma * np.log(1 - s0 + s0 * np.exp(2 * T))
    assert abs(uh[0, 0] - np.sqrt(s) * np.exp(1j * th)) < 1e-9
    assert np.max(np.abs(uh.ravel()[1:])) < 1e-15


def test_linear_part_multiplier():
    # with a negligible amplitude each mode is multiplied by sum_{p<=4} (L dt)^p / p! (RK4)
    # or exactly exp(L dt) (integrating factor).
    M, beta, gamma, dt = 8, 1.5, -0.5, 0.05
    g = np.random.default_rng(0)
    uh = 1e-9 * (g.standard_normal((M, M)) + 1j * g.standard_normal((M, M)))
    z = gl.linear_symbol(M, beta) * dt
    rk = gl.rk4_step(uh, dt, beta, gamma)
    assert np.max(np.abs(rk - uh * (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24))) < 1e-22
    ifr = gl.if_rk4_step(uh, dt, beta, gamma)
    assert np.max(np.abs(ifr - uh * np.exp(z))) < 1e-22


@pytest.mark.parametrize("M,factor", [(6, 1.5), (8, 1.5), (6, 2.0), (7, 1.5)])
def test_padded_product_equals_modular_convolution(M, factor):
    # The padded cubic term equals sum over a + b - c == m (mod Mp) of u_a u_b conj(u_c):
    # with factor 2 (Mp >= 2M) no sum wraps, i.e. exact de-aliasing; with 3/2 the
    # wrapped terms are exactly those the padded mesh aliases.
    g = np.random.default_rng(1)
    uh = g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))
    Mp = {1.5: 3 * M // 2, 2.0: 2 * M}[factor]           # the 3/2 rule's mesh (Sec. 6), or 2M
    assert gl.padded_size(M, factor) == Mp
    got = gl.nonlinear(uh, 0.0, factor)
    l = fourier.wavenumbers(M).astype(int)
    acc = {}
    for (i0, a0), (j0, b0), (k0, c0) in itertools.product(enumerate(l), repeat=3):
        for (i1, a1), (j1, b1), (k1, c1) in itertools.product(enumerate(l), repeat=3):
            key = ((a0 + b0 - c0) % Mp, (a1 + b1 - c1) % Mp)
            acc[key] = acc.get(key, 0) + uh[i0, i1] * uh[j0, j1] * np.conj(uh[k0, k1])
            if factor >= 2:
                assert abs(a0 + b0 - c0) < Mp and abs(a1 + b1 - c1) < Mp
    expect = np.array([[acc.get((a % Mp, b % Mp), 0) for b in l] for a in l])
    assert np.max(np.abs(got - expect)) < 1e-11 * np.max(np.abs(expect))


def test_symmetry_of_real_initial_condition():
    # Sec. 6: the real initial condition (x + y) exp(-0.03 (x^2 + y^2)) keeps u(x, y) = u(y, x)
    # when the nonlinear term is de-aliased (paper form beta = 0, gamma = 1.5).
    M = 20
    x, y = _grid(M)
    u0 = (x + y) * np.exp(-0.03 * (x ** 2 + y ** 2))
    uh = fourier.c2c_forward(fourier.c2c_forward(u0.astype(complex), 0), 1)
    for _ in range(20):
        uh = gl.rk4_step(uh, 0.025, 0.0, 1.5)
    assert np.max(np.abs(uh - uh.T)) < 1e-13 * np.max(np.abs(uh))
