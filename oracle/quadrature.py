"""Gauss quadrature and Shen basis values (oracle, test infrastructure).

Chebyshev family, Sec. 3.4.2 of the paper: the Chebyshev-Gauss points
x_j = cos((2j+1) pi / (2N)) and the constant weights w_j = pi / N, and the Shen
composite bases
  Dirichlet   phi_l = T_l - T_{l+2},                                   l = 0..N-3  (Eq. chebdirichlet)
  Neumann     phi_l = T_l - (l/(l+2))^2 T_{l+2},                       l = 0..N-3
              (Sec. 3.1 lists ShenNeumannBasis without its formula; this is Shen's
              Neumann basis, the combination with phi_l'(+-1) = 0, since T_n'(+-1) = (+-1)^(n+1) n^2)
  biharmonic  phi_l = T_l - 2(l+2)/(l+3) T_{l+2} + (l+1)/(l+3) T_{l+4}, l = 0..N-5  (Eq. chebbiharmonic)
  regular     phi_l = T_l,                                             l = 0..N-1
Legendre family (Sec. 3.1 lists the bases; Sec. 3.4.2 and Sec. 4 give the composite ones): the
Legendre-Gauss points and weights (weight function 1), taken in descending order like the
Chebyshev points, and
  Dirichlet   phi_l = L_l - L_{l+2}                                    (Eq. legdirichlet)
  biharmonic  phi_l = L_l - 2(2l+5)/(2l+7) L_{l+2} + (2l+3)/(2l+7) L_{l+4}  (Eq. legbiharmonic; the
              printed formula lacks the factor L_{l+4} of its last term, and this is the only
              completion for which phi_l and phi_l' vanish at x = +-1)
  regular     phi_l = L_l.
Basis values and derivatives are evaluated with NumPy's Chebyshev and Legendre series
routines (Clenshaw evaluation, coefficient-space differentiation); the Legendre-Gauss rule is
NumPy's leggauss.
"""
import numpy as np
from numpy.polynomial import chebyshev as npcheb
from numpy.polynomial import legendre as npleg

CHEBYSHEV_KINDS = ("chebyshev", "dirichlet", "neumann", "biharmonic")
LEGENDRE_KINDS = ("legendre", "legendre_dirichlet", "legendre_biharmonic")
KINDS = CHEBYSHEV_KINDS + LEGENDRE_KINDS


def family(kind):
    """"chebyshev" or "legendre": the orthogonal family a basis is built from."""
    return "legendre" if kind in LEGENDRE_KINDS else "chebyshev"


def regular_kind(kind):
    """The regular (orthogonal) basis of the family of ``kind``."""
    return "legendre" if kind in LEGENDRE_KINDS else "chebyshev"


def gauss_points(N):
    """Chebyshev-Gauss points and weights (Sec. 3.4.2, Chebyshev quadrature rule)."""
    j = np.arange(N, dtype=np.float64)
    x = np.cos((2.0 * j + 1.0) * np.pi / (2.0 * N))
    w = np.full(N, np.pi / N)
    return x, w


def legendre_points(N):
    """Legendre-Gauss points (descending) and weights: exact for degree <= 2N - 1, weight 1."""
    x, w = npleg.leggauss(N)
    return x[::-1].copy(), w[::-1].copy()


def points(kind, N):
    """Quadrature points and weights of the family of ``kind``."""
    return legendre_points(N) if family(kind) == "legendre" else gauss_points(N)


def num_basis(kind, N):
    """Number of basis functions: N, N-2 (index set l^D) or N-4 (index set l^B)."""
    return {"chebyshev": N, "dirichlet": N - 2, "neumann": N - 2, "biharmonic": N - 4,
            "legendre": N, "legendre_dirichlet": N - 2, "legendre_biharmonic": N - 4}[kind]


def basis_coefficients(kind, N):
    """Matrix P with phi_l = sum_k P[l, k] T_k (or L_k for the Legendre family), shape (num_basis, N)."""
    nb = num_basis(kind, N)
    P = np.zeros((nb, N))
    for l in range(nb):
        P[l, l] = 1.0
        if kind in ("dirichlet", "legendre_dirichlet"):
            P[l, l + 2] = -1.0
        elif kind == "neumann":
            P[l, l + 2] = -(l / (l + 2.0)) ** 2
        elif kind == "biharmonic":
            P[l, l + 2] = -2.0 * (l + 2) / (l + 3)
            P[l, l + 4] = (l + 1) / (l + 3)
        elif kind == "legendre_biharmonic":
            P[l, l + 2] = -2.0 * (2 * l + 5) / (2 * l + 7)
            P[l, l + 4] = (2 * l + 3) / (2 * l + 7)
    return P


def basis_values(kind, N, x, deriv=0):
    """V[j, l] = d^deriv phi_l / dx^deriv evaluated at x_j.

    The T- (or L-) coefficients of phi_l, differentiated in coefficient space, are summed
    against the Vandermonde matrix T_k(x_j) (or L_k(x_j)) of the three-term recurrence.
    """
    if family(kind) == "legendre":
        der, vander = npleg.legder, npleg.legvander
    else:
        der, vander = npcheb.chebder, npcheb.chebvander
    coef = basis_coefficients(kind, N).T         # (N, nb): one series per column
    if deriv:
        coef = der(coef, m=deriv, axis=0)
    x = np.asarray(x, dtype=np.float64)
    return vander(x, coef.shape[0] - 1) @ coef
