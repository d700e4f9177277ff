"""Galerkin matrices by brute-force quadrature, and dense solves (oracle).

Sec. 3.4.2 of the paper defines, with the discrete inner product of Eq. (quadrature),
  mass        B_ml = (phi_l, phi_m)_w^N
  stiffness   A_ml = (phi_l'', phi_m)_w^N
and Sec. 4 (biharmonic problem) adds
  bi-harmonic S_ml = (phi_l'''', phi_m)_w^N.
Row index m is the test function, column index l the trial function.  Each entry
is the quadrature sum over the N Gauss points of the basis' family (Chebyshev-Gauss,
or Legendre-Gauss with weight 1); nothing is taken from a closed form.

For one Fourier column with squared wavenumber kappa2 (Eq. laplace), the weak
forms of
  a lap(u) + b u = f                       ->  (a (A - kappa2 B) + b B) u_hat = S(f)
  a lap^2(u) + b lap(u) + c u = f          ->  (a (S - 2 kappa2 A + kappa2^2 B)
                                                + b (A - kappa2 B) + c B) u_hat = S(f)
after dividing both sides by the common Fourier factor (2 pi per periodic axis,
or its domain length), are solved here by dense LU.
"""
import functools

import numpy as np

from . import quadrature


@functools.lru_cache(maxsize=32)
def _matrix(kind, N, q):
    """[m, l] = sum_j phi_m(x_j) w_j phi_l^(q)(x_j), the quadrature of (phi_l^(q), phi_m)_w^N."""
    x, w = quadrature.points(kind, N)
    phi = quadrature.basis_values(kind, N, x, 0)          # (N, nb)
    dphi = quadrature.basis_values(kind, N, x, q)
    m = (phi * w[:, None]).T @ dphi
    m.setflags(write=False)
    return m


class _Matrices(dict):
    """B, A, S computed on first access (each an independent quadrature)."""

    def __init__(self, kind, N):
        super().__init__()
        self.kind, self.N = kind, N

    def __missing__(self, name):
        value = _matrix(self.kind, self.N, {"B": 0, "A": 2, "S": 4}[name])
        self[name] = value
        return value


def matrices(kind, N):
    """Dense B, A, S for the basis ``kind`` with N quadrature points (computed when first used)."""
    return _Matrices(kind, N)


def helmholtz_matrix(mats, a, b, kappa2):
    return a * (mats["A"] - kappa2 * mats["B"]) + b * mats["B"]


def biharmonic_matrix(mats, a, b, c, kappa2):
    B, A, S = mats["B"], mats["A"], mats["S"]
    return a * (S - 2.0 * kappa2 * A + kappa2 * kappa2 * B) + b * (A - kappa2 * B) + c * B


def solve_columns(kind, N, rhs, kappa2, system, singular=None):
    """Solve system(kappa2) u = rhs along axis 0 for every column.

    rhs has shape (N, ...) with the valid entries in rows 0..nb-1; kappa2 has
    the shape of rhs[0].  Rows nb..N-1 of the result are zero.

    singular(kappa2) -> bool marks columns whose system has the constant phi_0 in its
    null space (the Neumann basis with no zeroth-order term): there u_hat_0 = 0 and the
    equation of the test function phi_0 (the compatibility condition) is dropped.
    """
    nb = quadrature.num_basis(kind, N)
    rhs = np.asarray(rhs)
    cols = rhs.reshape(N, -1)
    k2 = np.broadcast_to(kappa2, rhs.shape[1:]).reshape(-1)
    out = np.zeros(cols.shape, dtype=np.result_type(cols.dtype, np.float64))
    for c in range(cols.shape[1]):
        M = system(k2[c])
        if singular is not None and singular(k2[c]):
            out[1:nb, c] = np.linalg.solve(M[1:, 1:], cols[1:nb, c])
        else:
            out[:nb, c] = np.linalg.solve(M, cols[:nb, c])
    return out.reshape(rhs.shape)
