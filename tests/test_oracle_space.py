"""Pins for the oracle's Fourier transforms and tensor-product space (CPU only)."""
import numpy as np
import pytest

from oracle import fourier
from oracle.space import Space
from paper_1708_03188_gb300 import inputs


def test_dft_single_mode_and_sign():
    # forward of exp(i l X) is a unit coefficient at wavenumber l (Sec. 3.4.1 definitions)
    M = 12
    X = 2 * np.pi * np.arange(M) / M
    for l in (-6, -5, -1, 0, 3, 5):
        uh = fourier.c2c_forward(np.exp(1j * l * X), 0)
        k = fourier.wavenumbers(M)
        expect = (k == l).astype(float)
        assert np.max(np.abs(uh - expect)) < 1e-13
    # r2c of cos(3X) + sin(2X): 1/2 at l=3, -i/2 at l=2
    u = np.cos(3 * X) + np.sin(2 * X)
    uh = fourier.r2c_forward(u, 0)
    e = np.zeros(M // 2 + 1, complex)
    e[3] = 0.5
    e[2] = -0.5j
    assert np.max(np.abs(uh - e)) < 1e-14


@pytest.mark.parametrize("M", [16, 17])
def test_r2c_round_trip_paper_example(M):
    # Sec. 3.1: R2C forward then backward returns the random input (N = 16); odd length too.
    u = inputs.rng("poisson2d", 7).random(M)
    assert np.allclose(fourier.c2r_backward(fourier.r2c_forward(u, 0), M, 0), u, rtol=0, atol=1e-13)
    # Parseval: sum |u|^2 / M = sum over the full spectrum of |u_hat|^2
    full = fourier.c2c_forward(u.astype(complex), 0)
    assert abs(np.sum(u ** 2) / M - np.sum(np.abs(full) ** 2)) < 1e-13


def test_fourier_poisson_paper_example():
    # Sec. 3.4.1: u = cos(4x), f = u'' on N = 32 points; u_hat = f_hat / (-l^2), l != 0.
    N = 32
    X = 2 * np.pi * np.arange(N) / N
    f = -16 * np.cos(4 * X)
    fh = fourier.r2c_forward(f, 0)
    l = fourier.wavenumbers(N, r2c=True)
    uh = np.zeros_like(fh)
    uh[1:] = fh[1:] / (-(l[1:] ** 2))
    assert np.allclose(fourier.c2r_backward(uh, N, 0), np.cos(4 * X), rtol=0, atol=1e-13)


def test_dirichlet_poisson_1d_paper_example():
    # Sec. 3.4.2, Fig. poisson1D_dirichlet: u = sin(pi x)(1 - x^2), solve u'' = f, N = 32.
    N = 32
    S = Space(["dirichlet"], [N])
    x = inputs.cheb_points(N)
    u = np.sin(np.pi * x) * (1 - x ** 2)
    f = -np.pi ** 2 * np.sin(np.pi * x) * (1 - x ** 2) - 4 * np.pi * x * np.cos(np.pi * x) - 2 * np.sin(np.pi * x)
    uh = S.helmholtz(1.0, 0.0, S.scalar_product(f))
    assert np.max(np.abs(S.backward(uh) - u)) < 1e-13


def test_poisson2d_paper_example_odd_fourier():
    # Sec. 4, Fig. poisson2D: u = (cos 4y + sin 2x)(1 - x^2) on N = (32, 33), lap(u) = f.
    N = (32, 33)
    S = Space(["dirichlet", "r2c"], N)
    x, y = inputs.mesh(["dirichlet", "r2c"], N)
    u = (np.cos(4 * y) + np.sin(2 * x)) * (1 - x ** 2)
    f = (-4 * np.sin(2 * x) * (1 - x ** 2) - 8 * x * np.cos(2 * x) - 2 * (np.cos(4 * y) + np.sin(2 * x))
         - 16 * np.cos(4 * y) * (1 - x ** 2))
    uh = S.helmholtz(1.0, 0.0, S.scalar_product(f))
    assert np.max(np.abs(S.backward(uh) - u)) < 1e-12


def test_poisson2d_manufactured():
    N = (32, 32)
    S = Space(["dirichlet", "r2c"], N)
    x, y = inputs.mesh(["dirichlet", "r2c"], N)
    uh = S.helmholtz(-1.0, 0.0, S.scalar_product(inputs.poisson2d_f(x, y)))
    assert np.max(np.abs(S.backward(uh) - inputs.poisson2d_u(x, y))) < 1e-12


def test_helmholtz_with_mass_term():
    # a lap(u) + b u = f with b != 0: u = (1 - x^2) exp(x) cos(2y)
    N = (28, 12)
    a, b = 0.7, -3.0
    S = Space(["dirichlet", "r2c"], N)
    x, y = inputs.mesh(["dirichlet", "r2c"], N)
    g = (1 - x ** 2) * np.exp(x)
    g2 = (-1 - 4 * x - x ** 2) * np.exp(x)            # g''
    u = g * np.cos(2 * y)
    f = a * (g2 - 4 * g) * np.cos(2 * y) + b * u
    uh = S.helmholtz(a, b, S.scalar_product(f))
    assert np.max(np.abs(S.backward(uh) - u)) < 1e-12


@pytest.mark.parametrize("kind", ["dirichlet", "biharmonic"])
def test_box3d_exact_coefficients(kind):
    # (1-x^2)^2 = 3/8 T0 - 1/2 T2 + 1/8 T4: Dirichlet coefficients (3/8, 0, -1/8),
    # biharmonic (3/8); sin y -> -i/2 at m = 1 and +i/2 at m = -1; cos 2z -> 1/2 at n = 2.
    N = (12, 8, 8)
    kinds = [kind, "c2c", "r2c"]
    S = Space(kinds, N)
    x, y, z = inputs.mesh(kinds, N)
    u = inputs.box3d_u(x, y, z)
    uh = S.forward(u)
    e = np.zeros(S.spectral_shape, complex)
    lead = [0.375, 0, -0.125] if kind == "dirichlet" else [0.375]
    for i, c in enumerate(lead):
        e[i, 1, 2] = c * (-0.5j) * 0.5
        e[i, -1, 2] = c * (0.5j) * 0.5
    assert np.max(np.abs(uh - e)) < 1e-14
    f = inputs.box3d_f_poisson(x, y, z) if kind == "dirichlet" else inputs.box3d_f_biharmonic(x, y, z)
    st = S.scalar_product(f)
    sol = S.helmholtz(-1.0, 0.0, st) if kind == "dirichlet" else S.biharmonic(1.0, 0.0, 0.0, st)
    assert np.max(np.abs(sol - e)) < 1e-14


@pytest.mark.parametrize("kinds,N", [(["dirichlet"], [16]), (["dirichlet", "r2c"], [10, 9]),
                                     (["biharmonic", "c2c", "r2c"], [12, 6, 8]),
                                     (["chebyshev", "c2c"], [9, 5])])
def test_round_trips(kinds, N):
    # Sec. 3.3: forward/backward is not the identity on raw data but is on the space.
    S = Space(kinds, N)
    g = inputs.rng("box3d", 3)
    raw = g.standard_normal(tuple(N))
    if not S.real:
        raw = raw + 1j * g.standard_normal(tuple(N))
    v = S.backward(S.forward(raw))
    assert np.max(np.abs(S.backward(S.forward(v)) - v)) < 1e-12
    if kinds[0] != "chebyshev":
        assert np.max(np.abs(v - raw)) > 1e-3
    c = S.forward(v)
    assert np.max(np.abs(S.forward(S.backward(c)) - c)) < 1e-12


def test_biharmonic_general_coefficients():
    # a lap^2 u + b lap u + c u = f with u = (1-x^2)^2 cos(3y) (clamped at x = +-1)
    N = (24, 10)
    a, b, c = 1.3, -0.4, 2.0
    S = Space(["biharmonic", "r2c"], N)
    x, y = inputs.mesh(["biharmonic", "r2c"], N)
    g = (1 - x ** 2) ** 2
    g2 = 12 * x ** 2 - 4
    g4 = 24 + 0 * x
    ky2 = 9.0
    lap = (g2 - ky2 * g)
    lap2 = g4 - 2 * ky2 * g2 + ky2 ** 2 * g
    f = (a * lap2 + b * lap + c * g) * np.cos(3 * y)
    uh = S.biharmonic(a, b, c, S.scalar_product(f))
    assert np.max(np.abs(S.backward(uh) - g * np.cos(3 * y))) < 1e-12
