"""Pins for the oracle's Legendre family (Sec. 3.1, Eq. legdirichlet, Eq. legbiharmonic; CPU only).

Routes independent of the oracle's quadrature and NumPy series code:
  - Legendre polynomials from Bonnet's recursion in exact rationals, and integrals of
    monomials over [-1, 1]: exact mass, stiffness and biharmonic matrices;
  - Shen's closed forms for the Legendre-Dirichlet basis;
  - the boundary conditions that fix the reading of the printed biharmonic basis;
  - manufactured solutions: the paper's 1-D Poisson example and (1 - x^2)^2 sin y cos 2z, whose
    Legendre coefficients are exact simple fractions.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import galerkin, quadrature
from oracle.space import Space
from paper_1708_03188_gb300 import inputs


def legendre_monomials(n_max):
    """L_0..L_{n_max} as lists of Fraction monomial coefficients (Bonnet's recursion)."""
    L = [[Fraction(1)], [Fraction(0), Fraction(1)]]
    for n in range(1, n_max):
        xl = [Fraction(0)] + L[n]
        prev = L[n - 1] + [Fraction(0)] * 2
        L.append([((2 * n + 1) * xl[i] - n * prev[i]) / (n + 1) for i in range(n + 2)])
    return L[: n_max + 1]


def padd(p, q, a=Fraction(1), b=Fraction(1)):
    n = max(len(p), len(q))
    p = p + [Fraction(0)] * (n - len(p))
    q = q + [Fraction(0)] * (n - len(q))
    return [a * u + b * v for u, v in zip(p, q)]


def pmul(p, q):
    out = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def pder(p, m=1):
    for _ in range(m):
        p = [i * p[i] for i in range(1, len(p))] or [Fraction(0)]
    return p


def integral(p):
    """int_{-1}^{1} p(x) dx, exactly."""
    return sum(Fraction(2, n + 1) * a for n, a in enumerate(p) if n % 2 == 0)


def basis_monomials(kind, N):
    L = legendre_monomials(N)
    out = []
    for l in range(quadrature.num_basis(kind, N)):
        p = L[l]
        if kind == "legendre_dirichlet":
            p = padd(p, L[l + 2], b=Fraction(-1))
        elif kind == "legendre_biharmonic":
            p = padd(padd(p, L[l + 2], b=Fraction(-2 * (2 * l + 5), 2 * l + 7)), L[l + 4],
                     b=Fraction(2 * l + 3, 2 * l + 7))
        out.append(p)
    return out


@pytest.mark.parametrize("N", [4, 9, 16])
def test_legendre_gauss_exactness_and_orthogonality(N):
    x, w = quadrature.legendre_points(N)
    assert np.all(np.diff(x) < 0)
    for n in range(2 * N):
        exact = 2.0 / (n + 1) if n % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** n) - exact) < 1e-14
    V = quadrature.basis_values("legendre", N, x)
    G = (V * w[:, None]).T @ V
    assert np.allclose(G, np.diag(2.0 / (2 * np.arange(N) + 1)), rtol=0, atol=1e-14)


@pytest.mark.parametrize("kind", ["legendre", "legendre_dirichlet", "legendre_biharmonic"])
@pytest.mark.parametrize("N", [8, 11])
def test_legendre_galerkin_matrices_equal_exact_rationals(kind, N):
    phis = basis_monomials(kind, N)
    mats = galerkin.matrices(kind, N)
    for name, q in (("B", 0), ("A", 2), ("S", 4)):
        exact = np.array([[float(integral(pmul(pder(pl, q), pm))) for pl in phis] for pm in phis])
        assert np.allclose(mats[name], exact, rtol=0, atol=1e-12 * max(1.0, np.abs(exact).max())), name


def test_legendre_dirichlet_closed_forms():
    N = 14
    mats = galerkin.matrices("legendre_dirichlet", N)
    k = np.arange(N - 2)
    B = np.diag(2 / (2 * k + 1) + 2 / (2 * k + 5))
    B += np.diag(-2 / (2 * k[:-2] + 5), 2) + np.diag(-2 / (2 * k[:-2] + 5), -2)
    assert np.allclose(mats["B"], B, rtol=0, atol=1e-14)
    assert np.allclose(mats["A"], -np.diag(4 * k + 6.0), rtol=0, atol=1e-12)    # diagonal stiffness


def test_legendre_biharmonic_reading_satisfies_the_boundary_conditions():
    N = 20
    for deriv in (0, 1):
        v = quadrature.basis_values("legendre_biharmonic", N, np.array([-1.0, 1.0]), deriv)
        assert np.max(np.abs(v)) < 1e-12, deriv
    # the formula as printed, with a constant (2l+3)/(2l+7) in place of (2l+3)/(2l+7) L_{l+4},
    # misses the Neumann condition: its derivative at x = 1 does not vanish
    leg = np.polynomial.legendre
    for l in range(1, 6):
        c = np.zeros(l + 3)
        c[l] = 1.0
        c[l + 2] = -2.0 * (2 * l + 5) / (2 * l + 7)
        c[0] += (2 * l + 3) / (2 * l + 7)
        assert abs(leg.legval(1.0, leg.legder(c))) > 1.0


def test_legendre_poisson_1d_paper_example():
    # Sec. 3.4.2: the Dirichlet Poisson example with the Legendre basis instead, u'' = f, N = 32
    N = 32
    S = Space(["legendre_dirichlet"], [N])
    x = inputs.legendre_points(N)
    u = np.sin(np.pi * x) * (1 - x ** 2)
    f = -np.pi ** 2 * np.sin(np.pi * x) * (1 - x ** 2) - 4 * np.pi * x * np.cos(np.pi * x) - 2 * np.sin(np.pi * x)
    uh = S.helmholtz(1.0, 0.0, S.scalar_product(f))
    assert np.max(np.abs(S.backward(uh) - u)) < 1e-13


@pytest.mark.parametrize("kind,cheb", [("legendre_dirichlet", [8 / 15, 0, -8 / 35]), ("legendre_biharmonic", [8 / 15])])
def test_legendre_box3d_exact_coefficients_and_solves(kind, cheb):
    # (1-x^2)^2 = 8/15 L_0 - 16/21 L_2 + 8/35 L_4 = 8/15 (L_0 - 10/7 L_2 + 3/7 L_4)
    N = (12, 8, 8)
    kinds = [kind, "c2c", "r2c"]
    sp = Space(kinds, N)
    x, y, z = inputs.mesh(kinds, N)
    u = np.broadcast_to(inputs.box3d_u(x, y, z), N)
    expect = np.zeros(sp.spectral_shape, complex)
    for k, c in enumerate(cheb):
        expect[k, 1, 2] = c * (-0.5j) * 0.5
        expect[k, -1, 2] = c * (0.5j) * 0.5
    assert np.max(np.abs(sp.forward(u) - expect)) < 1e-14
    if kind == "legendre_dirichlet":
        uh = sp.helmholtz(-1.0, 0.0, sp.scalar_product(np.broadcast_to(inputs.box3d_f_poisson(x, y, z), N)))
    else:
        uh = sp.biharmonic(1.0, 0.0, 0.0, sp.scalar_product(np.broadcast_to(inputs.box3d_f_biharmonic(x, y, z), N)))
    assert np.max(np.abs(uh - expect)) < 1e-13


@pytest.mark.parametrize("kind", ["legendre", "legendre_dirichlet", "legendre_biharmonic"])
def test_legendre_round_trip_and_projected_derivative(kind):
    N = 13
    sp = Space([kind], [N])
    g = inputs.rng("box3d", 77)
    nb = quadrature.num_basis(kind, N)
    c = np.zeros(N)
    c[:nb] = g.standard_normal(nb)
    assert np.allclose(sp.forward(sp.backward(c)), c, rtol=0, atol=1e-13)
    # d/dx onto the regular Legendre basis: exact Legendre coefficients of p' for p = sum c_l phi_l
    phis = basis_monomials(kind, N)
    p = [Fraction(0)]
    for cl, pl in zip(c[:nb], phis):
        p = padd(p, pl, b=Fraction(float(cl)))
    L = legendre_monomials(N)
    for m in range(3):
        dp = pder(p, m) + [Fraction(0)] * N
        coef = [Fraction(0)] * N                  # monomials -> Legendre, top degree down
        for n in range(N - 1, -1, -1):
            coef[n] = dp[n] / L[n][n]
            dp = padd(dp, L[n], b=-coef[n])
        got = sp.project_dx(c, 0, m)
        exact = np.array([float(v) for v in coef])
        assert np.max(np.abs(got - exact)) < 1e-11 * max(1.0, np.abs(exact).max()), m
