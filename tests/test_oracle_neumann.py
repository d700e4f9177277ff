"""Pins for the oracle's Shen Neumann basis phi_l = T_l - (l/(l+2))^2 T_{l+2} (Sec. 3.1 lists
ShenNeumannBasis; the formula is Shen's) and its solves (CPU only).

Independent routes:
  - the boundary conditions phi_l'(+-1) = 0 from T_n'(+-1) = (+-1)^(n+1) n^2, in exact arithmetic;
  - the Galerkin matrices against closed forms derived by hand from (T_n'', T_m)_w =
    pi/2 n (n^2 - m^2) (m < n, same parity) and (T_m, T_m)_w = pi/2 c_m:
      B_kk = pi/2 (c_k + q_k^2),  B_{k,k+2} = B_{k+2,k} = -pi/2 q_k,      q_k = (k/(k+2))^2,
      A_kk = -2 pi k^2 (k+1)/(k+2),  A_kj = -4 pi (k+1) j^2 / (k+2)^2 (j > k, same parity),
    rows = test functions, columns = trial functions;
  - manufactured solutions with phi'(+-1) = 0: u = cos(pi x) (its Chebyshev series converges to
    round-off at N = 32), with kappa2 > 0 or a zeroth-order term (nonsingular systems);
  - the singular column (b - a kappa2 = 0): u_hat_0 = 0 and every other Galerkin equation holds.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import galerkin, quadrature
from oracle.space import Space


def test_neumann_basis_has_zero_boundary_derivatives():
    for N in (6, 11, 20):
        P = quadrature.basis_coefficients("neumann", N)
        for l in range(N - 2):
            for x in (1, -1):
                # T_n'(x) = x^(n+1) n^2 at x = +-1, exactly
                d = sum(Fraction(P[l, n]).limit_denominator(10 ** 6) * Fraction(x) ** (n + 1) * n * n
                        for n in range(N) if P[l, n] != 0)
                assert d == 0, (N, l, x)
        V = quadrature.basis_values("neumann", N, np.array([-1.0, 1.0]), deriv=1)
        assert np.max(np.abs(V)) < 1e-10 * N ** 2


@pytest.mark.parametrize("N", [8, 13])
def test_neumann_galerkin_matrices_closed_forms(N):
    mats = galerkin.matrices("neumann", N)
    nb = N - 2
    B = np.zeros((nb, nb))
    A = np.zeros((nb, nb))
    q = [(k / (k + 2.0)) ** 2 for k in range(nb)]
    for k in range(nb):
        ck = 2.0 if k == 0 else 1.0
        B[k, k] = np.pi / 2 * (ck + q[k] ** 2)
        if k + 2 < nb:
            B[k, k + 2] = B[k + 2, k] = -np.pi / 2 * q[k]
        A[k, k] = -2 * np.pi * k * k * (k + 1) / (k + 2)
        for j in range(k + 2, nb, 2):
            A[k, j] = -4 * np.pi * (k + 1) * j * j / (k + 2) ** 2
    assert np.allclose(mats["B"], B, rtol=0, atol=1e-12)
    assert np.allclose(mats["A"], A, rtol=0, atol=1e-10 * N ** 3)


def test_neumann_helmholtz_manufactured_1d():
    # -u'' + u = f, u = cos(pi x): u'(+-1) = 0, f = (pi^2 + 1) cos(pi x)
    N = 32
    sp = Space(["neumann"], [N])
    x, _ = quadrature.gauss_points(N)
    f = (np.pi ** 2 + 1) * np.cos(np.pi * x)
    u = sp.backward(sp.helmholtz(-1.0, 1.0, sp.scalar_product(f)))
    assert np.max(np.abs(u - np.cos(np.pi * x))) < 1e-13


def test_neumann_poisson_manufactured_2d():
    # -lap u = f, u = cos(pi x) sin(2y): kappa2 = 4 in the only excited columns
    N, M = 32, 16
    sp = Space(["neumann", "r2c"], [N, M])
    x, _ = quadrature.gauss_points(N)
    y = 2 * np.pi * np.arange(M) / M
    u = np.cos(np.pi * x)[:, None] * np.sin(2 * y)[None, :]
    f = (np.pi ** 2 + 4) * u
    got = sp.backward(sp.helmholtz(-1.0, 0.0, sp.scalar_product(f)))
    assert np.max(np.abs(got - u)) < 1e-13


def test_neumann_singular_column_reading():
    # the constant Fourier column of a pure Poisson problem: u_hat_0 = 0, and the Galerkin
    # equations of phi_1 .. phi_{N-3} hold
    N = 16
    sp = Space(["neumann", "r2c"], [N, 8])
    g = np.random.default_rng(3)
    f = g.standard_normal((N, 8))
    S = sp.scalar_product(f)
    uh = sp.helmholtz(-1.0, 0.0, S)
    assert np.all(uh[0, 0] == 0)
    M = galerkin.helmholtz_matrix(galerkin.matrices("neumann", N), -1.0, 0.0, 0.0)
    res = M @ uh[:N - 2, 0] - S[:N - 2, 0]
    assert np.max(np.abs(res[1:])) < 1e-12 * np.max(np.abs(S[:, 0]))
