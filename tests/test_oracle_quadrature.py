"""Pins for the oracle's quadrature, bases and Galerkin matrices (CPU only)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import galerkin, quadrature

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [4, 7, 8, 16, 33])
def test_gauss_chebyshev_exact_for_even_monomials(N):
    # int_{-1}^{1} x^(2m) / sqrt(1-x^2) dx = pi (2m-1)!! / (2m)!!, exact for 2m <= 2N-1.
    x, w = quadrature.gauss_points(N)
    for m in range(N):
        exact = math.pi
        for i in range(1, m + 1):
            exact *= (2 * i - 1) / (2 * i)
        assert abs(np.sum(w * x ** (2 * m)) - exact) < 1e-13 * max(1.0, exact)


@pytest.mark.parametrize("N", [6, 9, 16])
def test_chebyshev_orthogonality(N):
    # (T_a, T_b)_w^N = pi/2 c_a delta_ab for a + b <= 2N - 1 (Sec. 3.4.2 quadrature rule).
    x, w = quadrature.gauss_points(N)
    T = quadrature.basis_values("chebyshev", N, x)
    G = (T * w[:, None]).T @ T
    expect = np.diag([math.pi] + [math.pi / 2] * (N - 1))
    assert np.max(np.abs(G - expect)) < 1e-13
    # values agree with cos(k arccos x), the definition of T_k
    assert np.max(np.abs(T - np.cos(np.outer(np.arccos(x), np.arange(N))))) < 1e-12


def test_mass_matrix_printed_in_paper():
    B = galerkin.matrices("dirichlet", 8)["B"]
    expect = np.zeros_like(B)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "mass_dirichlet_N8.txt"))
            if ln.strip() and not ln.startswith("#")]
    fixed = set()
    for off, val in rows:
        if ":" in off:
            o, i = map(int, off.split(":"))
            expect[i, i + o] = float(val)
            fixed.add((i, i + o))
    for off, val in rows:
        if ":" in off:
            continue
        o = int(off)
        for i in range(B.shape[0]):
            j = i + o
            if 0 <= j < B.shape[1] and (i, j) not in fixed:
                expect[i, j] = float(val)
    assert np.max(np.abs(B - expect)) < 6e-9          # printed to 8 decimals


# ---- exact rational Galerkin entries, independent of quadrature and NumPy's series code ----
def _cheb_derivative(c):
    """Exact coefficients of d/dx sum c_k T_k (textbook recurrence, Fractions)."""
    n = len(c)
    d = [Fraction(0)] * n
    for k in range(n - 1, 0, -1):
        d[k - 1] = (d[k + 1] if k + 1 < n else Fraction(0)) + 2 * k * c[k]
    d[0] = d[0] / 2
    return d


def _exact_matrix(kind, N, q):
    """[m, l] = (phi_l^(q), phi_m)_w / pi using (T_a, T_b)_w = pi/2 c_a delta_ab exactly."""
    nb = quadrature.num_basis(kind, N)

    def coeffs(l):
        c = [Fraction(0)] * (N + 4)
        c[l] = Fraction(1)
        if kind == "dirichlet":
            c[l + 2] = Fraction(-1)
        elif kind == "biharmonic":
            c[l + 2] = Fraction(-2 * (l + 2), l + 3)
            c[l + 4] = Fraction(l + 1, l + 3)
        return c

    M = np.zeros((nb, nb))
    for l in range(nb):
        d = coeffs(l)
        for _ in range(q):
            d = _cheb_derivative(d)
        for m in range(nb):
            cm = coeffs(m)
            s = sum(d[a] * cm[a] * (Fraction(1) if a == 0 else Fraction(1, 2)) for a in range(N + 4))
            M[m, l] = float(s)
    return M


@pytest.mark.parametrize("kind,N", [("dirichlet", 6), ("dirichlet", 10), ("biharmonic", 8), ("biharmonic", 11)])
def test_galerkin_matrices_equal_exact_rationals(kind, N):
    mats = galerkin.matrices(kind, N)
    for name, q in (("B", 0), ("A", 2), ("S", 4)):
        exact = math.pi * _exact_matrix(kind, N, q)
        scale = max(1.0, np.max(np.abs(exact)))
        assert np.max(np.abs(mats[name] - exact)) < 1e-12 * scale, name


def test_dirichlet_stiffness_closed_form():
    # Shen's Chebyshev-Dirichlet stiffness: -A_kk = 2 pi (k+1)(k+2), -A_kj = 4 pi (k+1) for j = k+2, k+4, ...
    N = 14
    A = galerkin.matrices("dirichlet", N)["A"]
    for k in range(N - 2):
        for j in range(N - 2):
            if j == k:
                e = -2 * math.pi * (k + 1) * (k + 2)
            elif j > k and (j - k) % 2 == 0:
                e = -4 * math.pi * (k + 1)
            else:
                e = 0.0
            assert abs(A[k, j] - e) < 1e-10 * (k + 1) ** 2


def test_biharmonic_structure():
    # S upper triangular with diagonal 8 pi (k+1)^2 (k+2)(k+4); A tridiagonal and B
    # pentadiagonal within each parity; odd offsets vanish.
    N = 20
    m = galerkin.matrices("biharmonic", N)
    nb = N - 4
    S, A, B = m["S"], m["A"], m["B"]
    for k in range(nb):
        assert abs(S[k, k] - 8 * math.pi * (k + 1) ** 2 * (k + 2) * (k + 4)) < 1e-9 * S[k, k]
    i, j = np.indices((nb, nb))
    assert np.max(np.abs(S[i > j])) < 1e-8
    assert np.max(np.abs(A[np.abs(i - j) > 2])) < 1e-8
    assert np.max(np.abs(B[np.abs(i - j) > 4])) < 1e-10
    for M in (S, A, B):
        assert np.max(np.abs(M[(i - j) % 2 == 1])) < 1e-8
