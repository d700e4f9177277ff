"""Chebyshev-Gauss quadrature and Shen basis values (oracle, test infrastructure).

Follows Sec. 3.4.2 of the paper: the Chebyshev-Gauss points
x_j = cos((2j+1) pi / (2N)) and the constant weights w_j = pi / N, and the Shen
composite bases
  Dirichlet   phi_l = T_l - T_{l+2},                                   l = 0..N-3  (Eq. chebdirichlet)
  biharmonic  phi_l = T_l - 2(l+2)/(l+3) T_{l+2} + (l+1)/(l+3) T_{l+4}, l = 0..N-5  (Eq. chebbiharmonic)
  regular     phi_l = T_l,                                             l = 0..N-1
Basis values and derivatives are evaluated with NumPy's Chebyshev series
routines (Clenshaw evaluation, coefficient-space differentiation).
"""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

KINDS = ("chebyshev", "dirichlet", "biharmonic")


def gauss_points(N):
    """Chebyshev-Gauss points and weights (Sec. 3.4.2, Chebyshev quadrature rule)."""
    j = np.arange(N, dtype=np.float64)
    x = np.cos((2.0 * j + 1.0) * np.pi / (2.0 * N))
    w = np.full(N, np.pi / N)
    return x, w


def num_basis(kind, N):
    """Number of basis functions: N, N-2 (index set l^D) or N-4 (index set l^B)."""
    return {"chebyshev": N, "dirichlet": N - 2, "biharmonic": N - 4}[kind]


def basis_coefficients(kind, N):
    """Matrix P with phi_l = sum_k P[l, k] T_k, shape (num_basis, N)."""
    nb = num_basis(kind, N)
    P = np.zeros((nb, N))
    for l in range(nb):
        P[l, l] = 1.0
        if kind == "dirichlet":
            P[l, l + 2] = -1.0
        elif kind == "biharmonic":
            P[l, l + 2] = -2.0 * (l + 2) / (l + 3)
            P[l, l + 4] = (l + 1) / (l + 3)
    return P


def basis_values(kind, N, x, deriv=0):
    """V[j, l] = d^deriv phi_l / dx^deriv evaluated at x_j.

    The T-coefficients of phi_l (differentiated in coefficient space) are summed against
    the Chebyshev Vandermonde matrix T_k(x_j) (three-term recurrence).
    """
    P = basis_coefficients(kind, N)
    coef = P.T                                   # (N, nb): one series per column
    if deriv:
        coef = npcheb.chebder(coef, m=deriv, axis=0)
    x = np.asarray(x, dtype=np.float64)
    V = npcheb.chebvander(x, coef.shape[0] - 1)  # (len(x), deg+1)
    return V @ coef
